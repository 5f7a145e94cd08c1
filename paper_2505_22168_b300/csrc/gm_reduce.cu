// gm_reduce.cu -- per-structure reductions and the force-matching loss.
//
//   E_i = sigma_Z (sum of output-layer partials + b3) + mu_Z      (Eq. scale_shift)
//   E_b = sum_{i in b} E_i                                       (Eq. energy_sum)
//   W_b = sum_{i in b} W_i (per-atom virials from the force kernel)
// Sums in 64-bit fixed point (exact, deterministic), returned as FP64.
//   loss (section "Training": energy and force terms, per-atom division of the energy term)
// One block per structure, fixed summation order (deterministic).
#include "gm_internal.h"
#include "gm_reduce.h"
#include "gm_fixed.cuh"

namespace gm {

__device__ __forceinline__ double block_sum_double(double v, double *sh) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) r += sh[q];
    return r;  // valid in thread 0
}

// One pass over the atoms: thread i forms E_i (and takes the per-atom virial) in FP32 and
// adds it to its structure's fixed-point accumulators (gm_fixed.cuh).  The block that
// finishes last (ticket counter after a device-scope fence, no waiting) converts the totals
// to FP64, writes energy and virial, and resets the accumulators and the counter.  The
// accumulators start from zero: the position-split kernel of the same step clears them.
__global__ void __launch_bounds__(REDUCE_CHUNK) k_reduce(int B, int N, const int32_t *__restrict__ atom_ptr,
                                                         const int32_t *__restrict__ species, int S,
                                                         const float *__restrict__ sigma, const float *__restrict__ mu,
                                                         const float *__restrict__ b3,
                                                         const float *__restrict__ nn_part, int nparts,
                                                         const float *__restrict__ vir_atom,
                                                         unsigned long long *acc, double *energy, double *virial) {
    __shared__ bool last;
    griddep_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31;
    const int nv = vir_atom ? 10 : 1;
    long long v[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) v[q] = 0;
    int b = -1;
    bool bad = false;
    if (i < N) {
        v[0] = to_fixed(atom_energy(i, species, S, sigma, mu, b3, nn_part, nparts), bad);
        if (vir_atom)
#pragma unroll
            for (int q = 0; q < 9; ++q) v[1 + q] = to_fixed(vir_atom[(size_t)i * 9 + q], bad);
        b = structure_of(atom_ptr, B, i);
    }
    warp_add_fixed<10>(b, v, nv, bad, acc, lane);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long ticket = atomicAdd(acc + (size_t)B * RW, 1ull);
        last = ticket == (unsigned long long)(gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    finalize_fixed(B, nv, acc, energy, virial, threadIdx.x, blockDim.x, [] { __syncthreads(); });
}

size_t reduce_acc_words(int B) { return (size_t)B * RW + 1; }

void launch_struct_reduce(int B, int N, const int32_t *atom_ptr, const int32_t *species, int S, const float *sigma,
                          const float *mu, const float *b3, const float *nn_part, int nparts, const float *vir_atom,
                          unsigned long long *acc, double *energy, double *virial, cudaStream_t st) {
    if (B <= 0) return;
    if (nparts < 2 || nparts > 16 || nparts % 2 != 0) {     // H in 64..512, a multiple of 64
        cudaMemsetAsync(energy, 0xff, sizeof(double) * B, st);   // NaN: not a supported width
        if (virial) cudaMemsetAsync(virial, 0xff, sizeof(double) * 9 * B, st);
        return;
    }
    if (N <= 0) {                                    // no atoms: every structure sums to zero
        cudaMemsetAsync(energy, 0, sizeof(double) * B, st);
        if (virial) cudaMemsetAsync(virial, 0, sizeof(double) * 9 * B, st);
        return;
    }
    launch_pdl(k_reduce, dim3((N + REDUCE_CHUNK - 1) / REDUCE_CHUNK), dim3(REDUCE_CHUNK), 0, st, B, N, atom_ptr, species,
               S, sigma, mu, b3, nn_part, nparts, vir_atom, acc, energy, virial);
    note_launches(1);
}

// Force-matching loss: one block; FP64 accumulation in a fixed order.
__global__ void __launch_bounds__(1024) k_loss(int B, int N, const int32_t *__restrict__ atom_ptr,
                                               const double *__restrict__ E, const double *__restrict__ Eref,
                                               const float *__restrict__ F, const float *__restrict__ Fref, double wE,
                                               double wF, double *loss, double *gE, float *gF) {
    __shared__ double sh[32];
    double le = 0.0, lf = 0.0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const double nb = (double)(atom_ptr[b + 1] - atom_ptr[b]);
        const double d = nb > 0.0 ? (E[b] - Eref[b]) / nb : 0.0;
        le += d * d;
        gE[b] = nb > 0.0 ? 2.0 * wE / B * d / nb : 0.0;
    }
    const double cF = N > 0 ? 2.0 * wF / (3.0 * N) : 0.0;
    for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) {
        const double d = (double)F[q] - (double)Fref[q];
        lf += d * d;
        gF[q] = (float)(cF * d);
    }
    const double se = block_sum_double(le, sh);
    __syncthreads();
    const double sf = block_sum_double(lf, sh);
    if (threadIdx.x == 0) *loss = wE / B * se + (N > 0 ? wF / (3.0 * N) * sf : 0.0);
}

void launch_loss(int B, int N, const int32_t *atom_ptr, const double *E, const double *Eref, const float *F,
                 const float *Fref, double wE, double wF, double *loss, double *gE, float *gF, cudaStream_t st) {
    k_loss<<<1, 1024, 0, st>>>(B, N, atom_ptr, E, Eref, F, Fref, wE, wF, loss, gE, gF);
    note_launches(1);
}

}  // namespace gm
