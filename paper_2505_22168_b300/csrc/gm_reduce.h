// gm_reduce.h -- FP64 per-structure reductions and the loss kernel.
#pragma once

#include "gm_internal.h"

namespace gm {

constexpr int REDUCE_CHUNK = 256;   // atoms per block (one per thread)
// accumulator words of launch_struct_reduce: [B][11] fixed-point sums and flags and a block counter, all
// zero before the launch (the kernel leaves them zero again)
size_t reduce_acc_words(int B);
void launch_struct_reduce(int B, int N, const int32_t *atom_ptr, const int32_t *species, int S, const float *sigma,
                          const float *mu, const float *b3, const float *nn_part, int nparts, const float *vir_atom,
                          unsigned long long *acc, double *energy, double *virial, cudaStream_t st);

void launch_loss(int B, int N, const int32_t *atom_ptr, const double *E, const double *Eref, const float *F,
                 const float *Fref, double wE, double wF, double *loss, double *gE, float *gF, cudaStream_t st);

}  // namespace gm
