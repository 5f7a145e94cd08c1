// gm_pair.h -- launchers of the per-pair kernels (moments, forces, parameter-gradient pair passes).
#pragma once

#include "gm_internal.h"

namespace gm {

struct PairArgs {
    int N, B, S;
    const int32_t *atom_ptr;
    const double *pos;
    const float4 *pos_hi, *pos_lo;   // hi/lo FP32 splits of pos (launch_split_pos)
    const int32_t *species;
    const double *cell;
    const int32_t *row_ptr;
    const int32_t *col;
    const char4 *shift;
    const float *beta;  // [S][S][NR][NB], pre-scaled by n_basis^{-1/2}
    RadialConst rc;
    int32_t *status;
};

// pos_hi[i] = (float)pos[i], pos_lo[i] = (float)(pos[i] - pos_hi[i]) per axis; pos_hi[i].w
// holds the bits of species[i] (lo w = 0).  zero_F [N][3] and zero_acc [n_acc], if not null,
// are cleared (the force kernel's and the structure reduction's accumulators).
void launch_split_pos(int N, const double *pos, const int32_t *species, float4 *hi, float4 *lo, float *zero_F,
                      unsigned long long *zero_acc, int n_acc, cudaStream_t st);
void launch_moments(const PairArgs &a, int tpa, float *psi, cudaStream_t st);
// heads > 1: the forces of that many shallow-ensemble heads in one launch, dpsi [heads][N][100]
// and F [heads][N][3] (vir_atom must be null)
void launch_forces(const PairArgs &a, int tpa, const float *dpsi, float *F, float *vir_atom, cudaStream_t st,
                   int heads = 1);

// parameter gradient: tangent moments along vel (= dL/dF) and block partials of dJ/dbeta
// tpa: lanes per atom as for launch_moments
void launch_moments_tangent(const PairArgs &a, int tpa, const float *vel, float *psid, cudaStream_t st);
int pg_beta_blocks(int N, int S);
void launch_pg_beta(const PairArgs &a, const float *vel, const float *psib, const float *psidb, float *part,
                    cudaStream_t st);

}  // namespace gm
