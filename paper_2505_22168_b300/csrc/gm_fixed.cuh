// gm_fixed.cuh -- per-structure sums in 64-bit fixed point (exact and deterministic).
//
//   E_i = sigma_Z (sum of output-layer partials + b3) + mu_Z      (Eq. scale_shift)
//   E_b = sum_{i in b} E_i                                       (Eq. energy_sum)
//
// Each value is converted to an integer in units of 2^-24 (the scaling by a power of two is
// exact; the rounding to the unit is below 3e-8 eV per atom).  Lanes of a warp that belong
// to the same structure add their integers with shuffles and one lane adds the result to
// the structure's accumulator with a 64-bit atomic.  Integer sums are exact, so the totals
// do not depend on the order of the atomics and equal the FP64 sum of the per-atom values to
// within the unit.  A value that is not finite or exceeds 1e9 in magnitude (a diverged
// model) is counted in an extra word per structure instead, and that structure's result
// comes out as NaN, as an FP64 sum would.  Accumulator layout per structure: energy, nine
// virial words, the NaN count (RW words); one ticket word after the last structure.
#pragma once

#include "gm_internal.h"

namespace gm {

constexpr float FIX_ONE = 16777216.0f;        // 2^24
constexpr double FIX_INV = 1.0 / 16777216.0;
constexpr int RW = 11;                         // accumulator words per structure

__device__ __forceinline__ long long to_fixed(float x, bool &bad) {
    if (!(fabsf(x) < 1e9f)) {
        bad = true;
        return 0;
    }
    return __float2ll_rn(x * FIX_ONE);
}

// E_i of atom i (< n_atoms) from its nparts output-layer partials (an even count, at most
// 16: H in 64..512), loaded together as float2 and added in order after b3
__device__ __forceinline__ float atom_energy(int i, const int32_t *species, int S, const float *sigma,
                                             const float *mu, const float *b3, const float *nn_part, int nparts) {
    float2 pt[8];
    const float2 *row = reinterpret_cast<const float2 *>(nn_part + (size_t)i * nparts);
#pragma unroll
    for (int t = 0; t < 8; ++t) pt[t] = 2 * t < nparts ? row[t] : make_float2(0.0f, 0.0f);
    float nn = b3[0];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        if (2 * t < nparts) {
            nn += pt[t].x;
            nn += pt[t].y;
        }
    }
    const int z = min(max(species[i], 0), S - 1);
    return fmaf(sigma[z], nn, mu[z]);
}

// Warp-level add of NV fixed-point values per lane (structure b, -1 for none) into the
// structures' accumulators: one round per structure present in the warp.
template <int NV>
__device__ __forceinline__ void warp_add_fixed(int b, const long long (&v)[NV], int nv, bool bad,
                                               unsigned long long *acc, int lane) {
    unsigned todo = __ballot_sync(0xffffffffu, b >= 0);
    while (todo) {
        const int lead = __ffs(todo) - 1;
        const int bl = __shfl_sync(0xffffffffu, b, lead);
        const bool mine = b == bl;
        todo &= ~__ballot_sync(0xffffffffu, mine);
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            if (q >= nv) break;
            long long x = mine ? v[q] : 0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            if (lane == lead) atomicAdd(acc + (size_t)bl * RW + q, (unsigned long long)x);
        }
        if (__any_sync(0xffffffffu, mine && bad) && lane == lead) atomicAdd(acc + (size_t)bl * RW + 10, 1ull);
    }
}

// Totals to FP64 (energy, and the virial when nv == 10), accumulators and ticket reset; by
// the nthr threads t of the block that took the last ticket (a barrier between the two loops
// is the caller's: bar() must synchronise exactly those threads)
template <typename Bar>
__device__ __forceinline__ void finalize_fixed(int B, int nv, unsigned long long *acc, double *energy, double *virial,
                                               int t, int nthr, Bar bar) {
    __threadfence();
    for (int q = t; q < B * 10; q += nthr) {
        const int s = q / 10, c = q - s * 10;
        if (c >= nv) continue;
        const long long x = (long long)atomicExch(acc + (size_t)s * RW + c, 0ull);
        const bool nan = atomicAdd(acc + (size_t)s * RW + 10, 0ull) != 0ull;
        const double val = nan ? __longlong_as_double(0x7ff8000000000000ll) : (double)x * FIX_INV;
        if (c == 0) energy[s] = val;
        else virial[9 * s + c - 1] = val;
    }
    bar();
    for (int s = t; s < B; s += nthr) atomicExch(acc + (size_t)s * RW + 10, 0ull);
    if (t == 0) atomicExch(acc + (size_t)B * RW, 0ull);
}

}  // namespace gm
