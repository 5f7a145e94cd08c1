// gm_ensemble.cu -- shallow-ensemble readout: per-head structure energies, their spread, and
// the spread of the per-head forces (section "Uncertainty Quantification").
//
// A shallow ensemble has E linear output heads on the same last hidden layer:
//   E_i^(k) = sigma_Z (w3e[k] . a2_i + b3e[k]) + mu_Z,  E^(k) = sum_i E_i^(k)
// and reports the mean over heads and the sample standard deviation with 1/E (Eq.
// uncertainty).  The forces are the gradient of the mean energy, which is one backward pass
// with the mean head (Eq. jacobian, left); in the Jacobian mode every head's forces F^(k) are
// evaluated as well (Eq. jacobian, right) and their spread per atom is reported.
#include "gm_ensemble.h"
#include "gm_fixed.cuh"

namespace gm {

size_t ens_acc_words(int B, int E) { return (size_t)B * (E + 1) + 1; }

// One thread per atom: the E head energies of atom i (from the L2 epilogue's partial sums
// nn_ens [E][nparts][ld], rows minor, added in order after b3e[k]) go to its structure's fixed-point
// accumulators (exact integer sums, as for the energy of the mean head).  The last block
// (ticket) converts the sums to FP64 and writes each structure's head energies, their mean's
// spread, and resets the accumulators.  Layout per structure: E sums, then a count of
// values outside the fixed-point range (the structure's results become NaN).
__global__ void __launch_bounds__(256) k_ens_energy(int B, int N, int E, const int32_t *__restrict__ atom_ptr,
                                                    const int32_t *__restrict__ species, int S,
                                                    const float *__restrict__ sigma, const float *__restrict__ mu,
                                                    const float *__restrict__ b3e, const float *__restrict__ nn_ens,
                                                    int nparts, size_t ld, unsigned long long *acc,
                                                    double *energy_heads, double *energy_std) {
    __shared__ bool last;
    griddep_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31;
    const int stride = E + 1;
    int b = -1;
    float sg = 0.0f, mz = 0.0f;
    if (i < N) {
        b = structure_of(atom_ptr, B, i);
        const int z = min(max(species[i], 0), S - 1);
        sg = sigma[z];
        mz = mu[z];
    }
    bool bad = false;
    for (int k = 0; k < E; ++k) {
        long long v = 0;
        if (i < N) {
            const float *col = nn_ens + (size_t)k * nparts * ld + i;
            float nn = b3e[k];
            for (int t = 0; t < nparts; ++t) nn += col[(size_t)t * ld];
            v = to_fixed(fmaf(sg, nn, mz), bad);
        }
        // one round per structure present in the warp (atoms of a structure are contiguous)
        unsigned todo = __ballot_sync(0xffffffffu, b >= 0);
        while (todo) {
            const int lead = __ffs(todo) - 1;
            const int bl = __shfl_sync(0xffffffffu, b, lead);
            const bool mine = b == bl;
            todo &= ~__ballot_sync(0xffffffffu, mine);
            long long x = mine ? v : 0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            if (lane == lead) atomicAdd(acc + (size_t)bl * stride + k, (unsigned long long)x);
        }
    }
    {   // values outside the fixed-point range: flag the structure
        unsigned todo = __ballot_sync(0xffffffffu, b >= 0);
        while (todo) {
            const int lead = __ffs(todo) - 1;
            const int bl = __shfl_sync(0xffffffffu, b, lead);
            const bool mine = b == bl;
            todo &= ~__ballot_sync(0xffffffffu, mine);
            if (__any_sync(0xffffffffu, mine && bad) && lane == lead) atomicAdd(acc + (size_t)bl * stride + E, 1ull);
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long ticket = atomicAdd(acc + (size_t)B * stride, 1ull);
        last = ticket == (unsigned long long)(gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (int s = threadIdx.x; s < B; s += blockDim.x) {
        const bool is_nan = atomicExch(acc + (size_t)s * stride + E, 0ull) != 0ull;
        double vals[GM_MAX_ENSEMBLE];
        double mean = 0.0;
        for (int k = 0; k < E; ++k) {
            vals[k] = (double)(long long)atomicExch(acc + (size_t)s * stride + k, 0ull) * FIX_INV;
            mean += vals[k];
        }
        mean /= (double)E;
        double var = 0.0;
        for (int k = 0; k < E; ++k) var += (vals[k] - mean) * (vals[k] - mean);
        if (energy_heads)
            for (int k = 0; k < E; ++k) energy_heads[(size_t)s * E + k] = is_nan ? nan : vals[k];
        if (energy_std) energy_std[s] = is_nan ? nan : sqrt(var / (double)E);
    }
    __syncthreads();
    if (threadIdx.x == 0) atomicExch(acc + (size_t)B * stride, 0ull);
}

// Per atom: the mean over heads of F^(k)_i and the spread
// sigma_F,i = sqrt(1/E sum_k |F^(k)_i - mean_k F^(k)_i|^2) (Eq. uncertainty with its implied
// sum over the three components).
__global__ void __launch_bounds__(256) k_ens_force_std(int N, int E, const float *__restrict__ Fk,
                                                       float *__restrict__ force_std) {
    griddep_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double m[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < E; ++k)
        for (int c = 0; c < 3; ++c) m[c] += (double)Fk[((size_t)k * N + i) * 3 + c];
    for (int c = 0; c < 3; ++c) m[c] /= (double)E;
    double var = 0.0;
    for (int k = 0; k < E; ++k)
        for (int c = 0; c < 3; ++c) {
            const double d = (double)Fk[((size_t)k * N + i) * 3 + c] - m[c];
            var += d * d;
        }
    force_std[i] = (float)sqrt(var / (double)E);
}

void launch_ens_energy(int B, int N, int E, const int32_t *atom_ptr, const int32_t *species, int S,
                       const float *sigma, const float *mu, const float *b3e, const float *nn_ens, int nparts,
                       size_t ld, unsigned long long *acc, double *energy_heads, double *energy_std,
                       cudaStream_t st) {
    if (B <= 0) return;
    if (N <= 0) {
        if (energy_heads) cudaMemsetAsync(energy_heads, 0, sizeof(double) * B * E, st);
        if (energy_std) cudaMemsetAsync(energy_std, 0, sizeof(double) * B, st);
        return;
    }
    launch_pdl(k_ens_energy, dim3((N + 255) / 256), dim3(256), 0, st, B, N, E, atom_ptr, species, S, sigma, mu, b3e,
               nn_ens, nparts, ld, acc, energy_heads, energy_std);
    note_launches(1);
}

void launch_ens_force_std(int N, int E, const float *Fk, float *force_std, cudaStream_t st) {
    if (N <= 0) return;
    launch_pdl(k_ens_force_std, dim3((N + 255) / 256), dim3(256), 0, st, N, E, Fk, force_std);
    note_launches(1);
}

}  // namespace gm
