// gm_ensemble.h -- shallow-ensemble readout kernels (gm_ensemble.cu).
#pragma once

#include "gm_internal.h"

namespace gm {

// accumulator words of launch_ens_energy: [B][E + 1] and a block counter, zero before the
// launch (the kernel leaves them zero again)
size_t ens_acc_words(int B, int E);
// head energies of every structure ([B][E], FP64) and their standard deviation over the
// heads ([B]); either output may be null
void launch_ens_energy(int B, int N, int E, const int32_t *atom_ptr, const int32_t *species, int S,
                       const float *sigma, const float *mu, const float *b3e, const float *nn_ens, int nparts,
                       size_t ld, unsigned long long *acc, double *energy_heads, double *energy_std,
                       cudaStream_t st);
// per-atom standard deviation over the heads of the forces Fk [E][N][3]
void launch_ens_force_std(int N, int E, const float *Fk, float *force_std, cudaStream_t st);

}  // namespace gm
