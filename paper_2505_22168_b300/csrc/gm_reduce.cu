// gm_reduce.cu -- per-structure FP64 reductions and the force-matching loss.
//
//   E_i = sigma_Z (sum of output-layer partials + b3) + mu_Z      (Eq. scale_shift)
//   E_b = sum_{i in b} E_i in FP64                               (Eq. energy_sum)
//   W_b = sum_{i in b} W_i in FP64 (per-atom virials from the force kernel)
// Sums run over fixed chunks of atoms and then over chunks in order (deterministic).
//   loss (section "Training": energy and force terms, per-atom division of the energy term)
// One block per structure, fixed summation order (deterministic).
#include "gm_internal.h"
#include "gm_reduce.h"

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

// Phase 1: block k takes atoms [k*CH, (k+1)*CH), one atom per thread: E_i (and the
// per-atom virial) go to shared memory, then one warp per structure overlapping the chunk
// sums its run and stores the partial at slot (b + k).  Consecutive chunks share at most
// one structure, so these slots never collide and structure b finds its partials at
// b + k for the chunks k it spans.  Phase 2 adds them in chunk order (deterministic).
__global__ void __launch_bounds__(REDUCE_CHUNK) k_reduce_partial(int B, int N, const int32_t *__restrict__ atom_ptr,
                                                                 const int32_t *__restrict__ species, int S,
                                                                 const float *__restrict__ sigma,
                                                                 const float *__restrict__ mu,
                                                                 const float *__restrict__ b3,
                                                                 const float *__restrict__ nn_part, int nparts,
                                                                 const float *__restrict__ vir_atom, double *part) {
    __shared__ float vals[10][REDUCE_CHUNK];
    const int k = blockIdx.x;
    const int c0 = k * REDUCE_CHUNK, c1 = min(N, c0 + REDUCE_CHUNK);
    const int i = c0 + threadIdx.x;
    if (i < c1) {
        float nn = b3[0];
        for (int t = 0; t < nparts; ++t) nn += nn_part[(size_t)i * nparts + t];
        const int z = min(max(species[i], 0), S - 1);
        vals[0][threadIdx.x] = fmaf(sigma[z], nn, mu[z]);
#pragma unroll
        for (int q = 0; q < 9; ++q) vals[1 + q][threadIdx.x] = vir_atom ? vir_atom[(size_t)i * 9 + q] : 0.0f;
    }
    __syncthreads();
    const int bf = structure_of(atom_ptr, B, c0), bl = structure_of(atom_ptr, B, c1 - 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int b = bf + warp; b <= bl; b += REDUCE_CHUNK / 32) {
        const int lo = max(atom_ptr[b], c0) - c0, hi = min(atom_ptr[b + 1], c1) - c0;
        double acc[10];
#pragma unroll
        for (int q = 0; q < 10; ++q) acc[q] = 0.0;
        for (int t = lo + lane; t < hi; t += 32)
#pragma unroll
            for (int q = 0; q < 10; ++q) acc[q] += (double)vals[q][t];
#pragma unroll
        for (int q = 0; q < 10; ++q)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc[q] += __shfl_down_sync(0xffffffffu, acc[q], off);
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < 10; ++q) part[(size_t)(b + k) * 10 + q] = acc[q];
    }
}

// Phase 2: one block per structure.  Lane l < 30 of warp w reads component l % 10 of chunks
// k0 + 3w + l / 10, k0 + 3w + l / 10 + 24, ...; the 24 running sums per component are then
// added in a fixed order (deterministic for a given structure size).
constexpr int RF_THREADS = 256, RF_LANES = 24;
__global__ void __launch_bounds__(RF_THREADS) k_reduce_final(int B, const int32_t *__restrict__ atom_ptr,
                                                             const double *__restrict__ part, double *energy,
                                                             double *virial) {
    __shared__ double sh[RF_LANES][10];
    const int b = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int a0 = atom_ptr[b], a1 = atom_ptr[b + 1];
    const int sub = warp * 3 + lane / 10, q = lane % 10;
    if (lane < 30) {
        double s = 0.0;
        if (a1 > a0)
            for (int k = a0 / REDUCE_CHUNK + sub; k <= (a1 - 1) / REDUCE_CHUNK; k += RF_LANES)
                s += part[(size_t)(b + k) * 10 + q];
        sh[sub][q] = s;
    }
    __syncthreads();
    if (threadIdx.x < 10) {
        double s = 0.0;
        for (int t = 0; t < RF_LANES; ++t) s += sh[t][threadIdx.x];
        if (threadIdx.x == 0) energy[b] = s;
        else if (virial) virial[9 * b + threadIdx.x - 1] = s;
    }
}

size_t reduce_partial_doubles(int B, int N) { return (size_t)(B + (N + REDUCE_CHUNK - 1) / REDUCE_CHUNK + 1) * 10; }

void launch_struct_reduce(int B, int N, const int32_t *atom_ptr, const int32_t *species, int S, const float *sigma,
                          const float *mu, const float *b3, const float *nn_part, int nparts, const float *vir_atom,
                          double *part, double *energy, double *virial, cudaStream_t st) {
    const int chunks = (N + REDUCE_CHUNK - 1) / REDUCE_CHUNK;
    if (chunks > 0) {
        k_reduce_partial<<<chunks, REDUCE_CHUNK, 0, st>>>(B, N, atom_ptr, species, S, sigma, mu, b3, nn_part, nparts, vir_atom,
                                                 part);
        note_launches(1);
    }
    if (B > 0) {
        k_reduce_final<<<B, RF_THREADS, 0, st>>>(B, atom_ptr, part, energy, virial);
        note_launches(1);
    }
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
