// gm_md.h -- molecular-dynamics kernels (gm_md.cu): velocity Verlet, Nose-Hoover chain,
// skin test for the neighbour list.
#pragma once

#include "gm_internal.h"

namespace gm {

// GM_OK or GM_ERR_ARG for the integration parameters
gm_status md_check_params(const gm_md_params *p);
// first thermostat half step of every structure (at the start of a run); pending[b] = its factor
void md_thermo(int B, const int32_t *atom_ptr, const gm_md_params &p, double *chain, double *kinetic,
               double *pending, const int32_t *status, cudaStream_t st);
// v = factor_b v + dt/2 F/m (factor may be null: 1); r += dt v; *flag = 1 if an atom moved more
// than skin/2 from pos_ref
void md_kick_drift(int N, int B, const int32_t *atom_ptr, const int32_t *species, const double *mass, const float *F,
                   const double *factor, const gm_md_params &p, double *vel, double *pos, const double *pos_ref,
                   int32_t *flag, const int32_t *status, cudaStream_t st);
// v += dt/2 F/m (if kick); pos_ref = pos when *flag; kinetic energies; NVT: second half step
// and, unless last_step, the next step's first (their velocity factor to pending); flag
// cleared and n_builds incremented when it was set.
// acc: reduce_acc_words(B) words, zero before the first launch (left zero)
void md_kick_ke(int N, int B, const int32_t *atom_ptr, const int32_t *species, const double *mass, const float *F,
                const gm_md_params &p, int kick, double *vel, const double *pos, double *pos_ref, int32_t *flag,
                unsigned long long *acc, double *kinetic, double *chain, double *pending, int64_t *n_builds,
                int last_step, const int32_t *status, cudaStream_t st);
// v *= pending_b (after the last step of a run)
void md_finish(int N, int B, const int32_t *atom_ptr, const double *pending, double *vel, const int32_t *status,
               cudaStream_t st);

}  // namespace gm
