// gm_common.cuh -- shared definitions of the libgm CUDA kernels (sm_103a).
//
// Moments are stored per atom as [n_radial = 5][20] FP32 unique components of the
// symmetric tensors Psi_{L,s} (Eq. basis_fn), L = 0..3:
//   c = 0        rank 0
//   c = 1..3     x y z
//   c = 4..9     xx xy xz yy yz zz
//   c = 10..19   xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
// Component c of rank L is the monomial ux^nx uy^ny uz^nz (nx+ny+nz = L) summed over
// neighbours with weight R_s.  A full-tensor entry Psi[a][b][c] equals the unique
// component with the same exponents, so full-tensor formulas read and write unique
// registers through idx2/idx3 (writes into the unique adjoint sum all permutations,
// which is exactly the gradient with respect to the unique component).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace gm {

constexpr int NR = 5;            // radial functions
constexpr int NB = 7;            // radial basis functions
constexpr int NC = 20;           // unique moment components per radial function
constexpr int NPSI = NR * NC;    // 100 moment values per atom
constexpr int NF = 360;          // invariant features (Eq. contraction, 8 families)
constexpr int NFP = 384;         // features padded to a multiple of 64
constexpr int MAX_S = 16;        // species
constexpr int TILE_M = 128;      // atom rows per GEMM tile

// exponent code nx*16 + ny*4 + nz of unique component c
__host__ __device__ constexpr int comp_code(int c) {
    switch (c) {
    case 0: return 0;
    case 1: return 16; case 2: return 4; case 3: return 1;
    case 4: return 32; case 5: return 20; case 6: return 17; case 7: return 8; case 8: return 5;
    case 9: return 2;
    case 10: return 48; case 11: return 36; case 12: return 33; case 13: return 24; case 14: return 21;
    case 15: return 18; case 16: return 12; case 17: return 9; case 18: return 6;
    default: return 3;
    }
}
__host__ __device__ constexpr int comp_nx(int c) { return comp_code(c) >> 4; }
__host__ __device__ constexpr int comp_ny(int c) { return (comp_code(c) >> 2) & 3; }
__host__ __device__ constexpr int comp_nz(int c) { return comp_code(c) & 3; }
__host__ __device__ constexpr int comp_rank(int c) { return c == 0 ? 0 : (c < 4 ? 1 : (c < 10 ? 2 : 3)); }

// tetrahedral and triangular numbers (closed forms keep every index a cheap constant)
__host__ __device__ constexpr int tri(int n) { return n * (n + 1) / 2; }
__host__ __device__ constexpr int tet(int n) { return n * (n + 1) * (n + 2) / 6; }
__host__ __device__ constexpr int imin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int imax(int a, int b) { return a < b ? b : a; }
// unique index of full rank-1/2/3 entries (sorted index tuples in lexicographic order)
__host__ __device__ constexpr int idx1(int a) { return 1 + a; }
__host__ __device__ constexpr int idx2(int a, int b) {
    return 4 + tri(3) - tri(3 - imin(a, b)) + (imax(a, b) - imin(a, b));
}
__host__ __device__ constexpr int idx3s(int a, int b, int c) {  // a <= b <= c
    return 10 + tet(3) - tet(3 - a) + tri(3 - a) - tri(3 - b) + (c - b);
}
__host__ __device__ constexpr int idx3(int a, int b, int c) {
    return idx3s(imin(imin(a, b), c), imax(imin(a, b), imin(imax(a, b), c)), imax(imax(a, b), c));
}

// ---------------------------------------------------------------- feature indexing
// Family-major; within a family lexicographic in (s1, s2, s3) subject to:
//   #1 s;  #2,#3,#4 s1<=s2;  #5 s1<=s2<=s3;  #6 s1<=s3;  #7 s1<=s2;  #8 free.
constexpr int FAM_OFF1 = 0, FAM_OFF2 = 5, FAM_OFF3 = 20, FAM_OFF4 = 35, FAM_OFF5 = 50,
              FAM_OFF6 = 85, FAM_OFF7 = 160, FAM_OFF8 = 235;

__host__ __device__ constexpr int pair_le_index(int s1, int s2) {  // s1 <= s2
    return tri(NR) - tri(NR - s1) + (s2 - s1);
}
__host__ __device__ constexpr int f5_index(int s1, int s2, int s3) {  // s1 <= s2 <= s3
    return tet(NR) - tet(NR - s1) + tri(NR - s1) - tri(NR - s2) + (s3 - s2);
}
__host__ __device__ constexpr int f6_index(int s1, int s2, int s3) {  // s1 <= s3
    return NR * (tri(NR) - tri(NR - s1)) + s2 * (NR - s1) + (s3 - s1);
}
__host__ __device__ constexpr int f7_index(int s1, int s2, int s3) {  // s1 <= s2
    return pair_le_index(s1, s2) * NR + s3;
}
__host__ __device__ constexpr int f8_index(int s1, int s2, int s3) { return (s1 * NR + s2) * NR + s3; }

// ---------------------------------------------------------------- dependent launch
// Wait for the predecessor kernels of a programmatic dependent launch (no-op otherwise).
// The next kernel is released implicitly as this grid's blocks exit: releasing it early
// (griddepcontrol.launch_dependents at the start) helped the 1536-atom step by 2 us but slowed
// multi-wave grids by up to 20 % on B300; releasing early only from grids of at most 296
// blocks gave the mixed 1536-atom step 0.7 us and cost the FP32 one 30 %.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---------------------------------------------------------------- status word
__device__ __forceinline__ void set_status(int32_t *st, int32_t code) {
    if (st) atomicCAS(st, 0, code);
}
__device__ __forceinline__ bool status_bad(const int32_t *st) {
    return st && *reinterpret_cast<const volatile int32_t *>(st) != 0;
}

// structure index of atom i: largest b with atom_ptr[b] <= i
__device__ __forceinline__ int structure_of(const int32_t *__restrict__ atom_ptr, int n_struct, int i) {
    int lo = 0, hi = n_struct - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(atom_ptr + mid) <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------- activations
// ACT: 0 = tanh, 1 = SiLU.  Returns phi(z); d1 = phi'(z).
template <int ACT>
__device__ __forceinline__ float act_fwd(float z, float &d1) {
    if (ACT == 0) {
        float t = tanhf(z);
        d1 = 1.0f - t * t;
        return t;
    } else {
        float s = 1.0f / (1.0f + expf(-z));
        d1 = s * (1.0f + z * (1.0f - s));
        return z * s;
    }
}
// phi, phi', phi'' (parameter-gradient tangent pass)
template <int ACT>
__device__ __forceinline__ float act_fwd2(float z, float &d1, float &d2) {
    if (ACT == 0) {
        float t = tanhf(z);
        d1 = 1.0f - t * t;
        d2 = -2.0f * t * d1;
        return t;
    } else {
        float s = 1.0f / (1.0f + expf(-z));
        d1 = s * (1.0f + z * (1.0f - s));
        d2 = s * (1.0f - s) * (2.0f + z * (1.0f - 2.0f * s));
        return z * s;
    }
}

// ---------------------------------------------------------------- radial part
// Model constants the pair kernels need (beta is pre-scaled by n_basis^{-1/2}).
// gamma_l2 = gamma log2(e) (rounded once from FP64), so Phi_k = 2^(-gamma_l2 t^2): the
// result carries the same argument-rounding error as exp(-gamma t^2), which dominates
// either way for the wide arguments (up to ~60) of the outer Gaussians.
enum { BASIS_GAUSSIAN = 0, BASIS_BESSEL = 1 };
struct RadialConst {
    float r_cut, inv_r_cut, pi_inv_r_cut, gamma, gamma_l2;
    float mu[NB];
    int basis;
    float bes_a[NB];   // Bessel-like basis: a_k, rounded once from FP64
};

// Bessel-like basis of Kocer et al.: f_k = a_k [j0((k+1) t) + j0((k+2) t)], t = pi r / r_cut,
// j0(x) = sin(x)/x, times the cosine cutoff.  One accurate sin/cos of t (sincospif), then
// sin(q t) and cos(q t) for q = 2..NB+1 by the Chebyshev recurrence
// sin((q+1) t) = 2 cos(t) sin(q t) - sin((q-1) t) (same for cos); d/dr j0(q t) = (cos(q t) - j0(q t)) / r.
template <bool DERIV>
__device__ __forceinline__ void bessel_basis(const RadialConst &rc, float r, float (&B)[NB], float (&dB)[NB]) {
    float s1, c1;
    sincospif(r * rc.inv_r_cut, &s1, &c1);
    const bool inside = r < rc.r_cut;
    const float fc = inside ? 0.5f * (c1 + 1.0f) : 0.0f;
    const float dfc = inside ? -0.5f * rc.pi_inv_r_cut * s1 : 0.0f;
    const float inv_t = 1.0f / (r * rc.pi_inv_r_cut);
    const float inv_r = rc.pi_inv_r_cut * inv_t;
    float j[NB + 1], dj[NB + 1];
    float sp = 0.0f, cp = 1.0f, sq = s1, cq = c1;
#pragma unroll
    for (int q = 1; q <= NB + 1; ++q) {
        j[q - 1] = sq * inv_t * (1.0f / (float)q);
        if (DERIV) dj[q - 1] = (cq - j[q - 1]) * inv_r;
        const float sn = fmaf(2.0f * c1, sq, -sp), cn = fmaf(2.0f * c1, cq, -cp);
        sp = sq;
        cp = cq;
        sq = sn;
        cq = cn;
    }
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        const float ph = rc.bes_a[k] * (j[k] + j[k + 1]);
        B[k] = fc * ph;
        if (DERIV) dB[k] = fmaf(dfc, ph, fc * rc.bes_a[k] * (dj[k] + dj[k + 1]));
    }
}

// 2^x by the hardware approximation (ex2.approx.ftz.f32: relative error about 2^-22, results
// below 2^-126 flushed to zero; a Gaussian that small adds nothing to R_s of order one)
__device__ __forceinline__ float ex2_ftz(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// f_c Phi_k (B) and optionally its r-derivative (dB) for the 7 Gaussians.  The cutoff's
// cosine and sine take the hardware approximation on [0, pi] (absolute error below 4e-7,
// against f_c and Phi of order one).
// BAS is the model's basis (a template parameter of the pair kernels, so each kernel holds
// the code of one basis only and keeps its register budget)
template <bool DERIV, int BAS>
__device__ __forceinline__ void radial_basis(const RadialConst &rc, float r, float (&B)[NB], float (&dB)[NB]) {
    if (BAS == BASIS_BESSEL) {
        bessel_basis<DERIV>(rc, r, B, dB);
        return;
    }
    float sp, cp;
    __sincosf(r * rc.pi_inv_r_cut, &sp, &cp);
    const bool inside = r < rc.r_cut;
    const float fc = inside ? 0.5f * (cp + 1.0f) : 0.0f;
    const float dfc = inside ? -0.5f * rc.pi_inv_r_cut * sp : 0.0f;
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        const float t = r - rc.mu[k];
        const float ph = ex2_ftz(-rc.gamma_l2 * (t * t));
        B[k] = fc * ph;
        if (DERIV) dB[k] = ph * fmaf(-2.0f * rc.gamma * t, fc, dfc);
    }
}

// Coefficient rows beta[zi][zj][s][0..6] staged in shared memory with a stride of BETA_ROW
// floats (16-byte aligned, two 16-byte loads per row; the stride of 12 spreads the rows
// over all bank groups).
constexpr int BETA_ROW = 12;
__device__ __forceinline__ void stage_beta(const float *__restrict__ beta, int S, float *sb) {
    const int n = S * S * NR * BETA_ROW;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const int row = q / BETA_ROW, k = q - row * BETA_ROW;
        sb[q] = k < NB ? beta[row * NB + k] : 0.0f;
    }
}
// R_s = sum_k beta[s][k] B_k (and R'_s from dB) for the five radial functions, from the
// staged rows of one species pair (bt = sb + (zi S + zj) NR BETA_ROW)
template <bool DERIV>
__device__ __forceinline__ void radial_combine(const float *bt, const float (&B)[NB], const float (&dB)[NB],
                                               float (&R)[NR], float (&Rp)[NR]) {
#pragma unroll
    for (int s = 0; s < NR; ++s) {
        const float4 c0 = *reinterpret_cast<const float4 *>(bt + s * BETA_ROW);
        const float4 c1 = *reinterpret_cast<const float4 *>(bt + s * BETA_ROW + 4);
        const float c[NB] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z};
        float v = 0.0f, w = 0.0f;
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            v = fmaf(c[k], B[k], v);
            if (DERIV) w = fmaf(c[k], dB[k], w);
        }
        R[s] = v;
        if (DERIV) Rp[s] = w;
    }
}

// the 20 monomials m_c(u) of the unit vector
__device__ __forceinline__ void monomials(float ux, float uy, float uz, float (&m)[NC]) {
    const float xx = ux * ux, yy = uy * uy, zz = uz * uz;
    m[0] = 1.0f;
    m[1] = ux; m[2] = uy; m[3] = uz;
    m[4] = xx; m[5] = ux * uy; m[6] = ux * uz; m[7] = yy; m[8] = uy * uz; m[9] = zz;
    m[10] = xx * ux; m[11] = xx * uy; m[12] = xx * uz; m[13] = ux * yy; m[14] = ux * uy * uz;
    m[15] = ux * zz; m[16] = yy * uy; m[17] = yy * uz; m[18] = uy * zz; m[19] = zz * uz;
}

// integer power for small exponents
__device__ __forceinline__ float ipow(float x, int n) {
    return n == 0 ? 1.0f : (n == 1 ? x : (n == 2 ? x * x : x * x * x));
}

// d m_c / d u_axis (axis 0, 1, 2); with constant c and axis it folds to a product
__device__ __forceinline__ float dmono(int c, int axis, float ux, float uy, float uz) {
    const int nx = comp_nx(c), ny = comp_ny(c), nz = comp_nz(c);
    if (axis == 0) return nx == 0 ? 0.0f : nx * ipow(ux, nx - 1) * ipow(uy, ny) * ipow(uz, nz);
    if (axis == 1) return ny == 0 ? 0.0f : ny * ipow(ux, nx) * ipow(uy, ny - 1) * ipow(uz, nz);
    return nz == 0 ? 0.0f : nz * ipow(ux, nx) * ipow(uy, ny) * ipow(uz, nz - 1);
}

}  // namespace gm
