// gm_contract.cu -- invariant features from the Gaussian moments (Eq. contraction) and
// the gradient of the energy with respect to the moments.
//
// Features (360 for 5 radial functions), family-major, lexicographic in (s1, s2, s3):
//   #1 Psi0_s                                  5
//   #2 Psi1_s1 . Psi1_s2              s1<=s2   15   (printed in Eq. contraction)
//   #3 Psi2_s1 : Psi2_s2              s1<=s2   15
//   #4 Psi3_s1 : Psi3_s2              s1<=s2   15
//   #5 (Psi2_s1)_ab (Psi2_s2)_bc (Psi2_s3)_ca  s1<=s2<=s3  35
//   #6 (Psi1_s1)_a (Psi2_s2)_ab (Psi1_s3)_b    s1<=s3      75
//   #7 (Psi3_s1)_abc (Psi3_s2)_abd (Psi2_s3)_cd s1<=s2     75
//   #8 (Psi1_s1)_a (Psi3_s2)_abc (Psi2_s3)_bc  all         125  (printed in Eq. contraction)
//
// Layout: a block holds 32 atoms (lane = atom) whose moments are staged in shared memory;
// its warps walk a list of work items (one family restricted to one radial index or index
// pair, see the item kernels below).  The 360 features of the 32 atoms are staged in shared
// memory and written as coalesced rows of the [M][384] GEMM operand (columns 360..383 are
// zero).  Backward: dE/dPsi over the unique components (100 per atom), with full-tensor
// index loops whose writes land in unique accumulators (this sums all index permutations,
// i.e. the gradient with respect to the unique component); per-warp partial gradients are
// added in warp order.  The parameter gradient runs the same items on dual numbers.
#include "gm_contract.h"

namespace gm {

constexpr int CT_ATOMS = 32;
constexpr int GT_STRIDE = NF + 1;

// Forward-mode dual number (value, derivative along a tangent direction).  The features
// are polynomials of the moments, so running the same item code on duals gives exact
// tangents (parameter gradient: dG along dPsi, and the second-order term of the adjoint).
struct Dual {
    float v, d;
};
__device__ __forceinline__ float mad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ Dual mad(Dual a, Dual b, Dual c) { return {fmaf(a.v, b.v, c.v), fmaf(a.d, b.v, fmaf(a.v, b.d, c.d))}; }
__device__ __forceinline__ Dual mad(float a, Dual b, Dual c) { return {fmaf(a, b.v, c.v), fmaf(a, b.d, c.d)}; }
__device__ __forceinline__ Dual mad(Dual a, float b, Dual c) { return {fmaf(a.v, b, c.v), fmaf(a.d, b, c.d)}; }
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual &operator+=(Dual &a, Dual b) { a.v += b.v; a.d += b.d; return a; }
__device__ __forceinline__ Dual &operator+=(Dual &a, float b) { a.v += b; return a; }
__device__ __forceinline__ Dual operator*(float a, Dual b) { return {a * b.v, a * b.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <typename T> __device__ __forceinline__ T zero();
template <> __device__ __forceinline__ float zero<float>() { return 0.0f; }
template <> __device__ __forceinline__ Dual zero<Dual>() { return {0.0f, 0.0f}; }

// feature stores: plain values to one tile row, duals to a value row and a tangent row
struct FeatOut {
    float *v, *d;
    __device__ __forceinline__ void put(int f, float x) const { v[f] = x; }
    __device__ __forceinline__ void put(int f, Dual x) const { v[f] = x.v; d[f] = x.d; }
};

// Stage the 360 leading columns of 32 rows of a [.][384] FP32 matrix into shared memory
// (row stride GT_STRIDE, rows past N zero).  Every thread issues all of its 16-byte loads
// before the first store, so the block waits for one memory latency instead of one per row.
template <int NT>
__device__ __forceinline__ void stage_rows(const float *__restrict__ src, int m0, int N, float *tile,
                                           bool tiled = false) {
    constexpr int V4 = NF / 4, TOT = CT_ATOMS * V4, PER = (TOT + NT - 1) / NT;
    // row-major [M][NFP], or the per-tile fused network kernel's layout: per 128-row tile,
    // 4-column groups major and rows minor (then consecutive threads take consecutive rows)
    float4 v[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int idx = threadIdx.x + u * NT;
        const int r = tiled ? idx % CT_ATOMS : idx / V4, q = tiled ? idx / CT_ATOMS : idx - r * V4;
        const int m = m0 + r;
        const size_t at = tiled ? (size_t)(m & ~127) * NFP + ((size_t)q * 128 + (m & 127)) * 4 : (size_t)m * NFP + 4 * q;
        v[u] = (idx < TOT && m < N) ? __ldg(reinterpret_cast<const float4 *>(src + at)) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int idx = threadIdx.x + u * NT;
        if (idx < TOT) {
            const int r = tiled ? idx % CT_ATOMS : idx / V4, q = tiled ? idx / CT_ATOMS : idx - r * V4;
            float *d = tile + r * GT_STRIDE + 4 * q;
            d[0] = v[u].x; d[1] = v[u].y; d[2] = v[u].z; d[3] = v[u].w;
        }
    }
    __syncthreads();
}

// ------------------------------------------------------------------ item kernels (FP32 path)
// The forward and backward kernels of the energy/force step stage the moments of 32 atoms
// in shared memory ([32][100], one row per atom; the 400-byte rows keep 16-byte accesses
// free of bank conflicts), lane = atom.  Every thread keeps the vectors and matrices of its
// atom (v_s, M_s: 45 values) in registers for the whole kernel; the rank-3 tensors T_s, and
// the one matrix an item selects at run time, are read from the shared tile.  The warps
// walk a list of 31 work items, each one family restricted to one radial index (or index
// pair) chosen at run time, with the other indices unrolled over the register tensors:
//   D(s1<=s2)  #7 and #4   15 items      E(s2)  #8   5 items      B(s1)  #5   5 items
//   C(s2)      #6          5 items       F      #1-#3  1 item
// Every item kind is one short loop body shared by all warps, so the instruction stream
// stays in the instruction cache (fully unrolled per-warp code, 15k FMAs per atom in the
// backward, starved the warps of instructions), and the shared-memory traffic is a few
// 16-byte accesses per item.  Items are dealt to the warps heaviest first in snake order.
// Backward: gradients with respect to v_s, M_s and Psi0_s accumulate in registers; those
// with respect to an item's run-time tensor (T_s1, T_s2; M_s1 in #5, M_s2 in #6) are added
// into the warp's private [32][100] shared slot (warp-private read-modify-write, no
// atomics), and the register sums join them at the end.  The slots are summed in warp order
// (deterministic).
constexpr int IT_COUNT = 31;
enum { IK_B = 0, IK_E = 1, IK_F = 2, IK_D = 3, IK_C = 4 };

#define LM(m, a, b) m[idx2(a, b) - 4]
#define LT(t, a, b, c) t[idx3(a, b, c) - 10]

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }

// Components of one radial channel (ch = row + s * 20, 16-byte aligned): 0 scalar, 1-3
// vector, 4-9 rank 2, 10-19 rank 3.
__device__ __forceinline__ void ld_v(const float *ch, float (&v)[3]) {
    const float4 q = ld4(ch);
    v[0] = q.y; v[1] = q.z; v[2] = q.w;
}
__device__ __forceinline__ void ld_m(const float *ch, float (&m)[6]) {
    const float4 a = ld4(ch + 4), b = ld4(ch + 8);
    m[0] = a.x; m[1] = a.y; m[2] = a.z; m[3] = a.w; m[4] = b.x; m[5] = b.y;
}
__device__ __forceinline__ void ld_t(const float *ch, float (&t)[10]) {
    const float4 a = ld4(ch + 8), b = ld4(ch + 12), c = ld4(ch + 16);
    t[0] = a.z; t[1] = a.w; t[2] = b.x; t[3] = b.y; t[4] = b.z; t[5] = b.w; t[6] = c.x; t[7] = c.y; t[8] = c.z;
    t[9] = c.w;
}
__device__ __forceinline__ void add_v(float *ch, const float (&v)[3], float c0) {
    float4 q = ld4(ch);
    q.x += c0; q.y += v[0]; q.z += v[1]; q.w += v[2];
    st4(ch, q);
}
__device__ __forceinline__ void add_m(float *ch, const float (&m)[6]) {
    float4 a = ld4(ch + 4), b = ld4(ch + 8);
    a.x += m[0]; a.y += m[1]; a.z += m[2]; a.w += m[3]; b.x += m[4]; b.y += m[5];
    st4(ch + 4, a);
    st4(ch + 8, b);
}
__device__ __forceinline__ void add_t(float *ch, const float (&t)[10]) {
    float4 a = ld4(ch + 8), b = ld4(ch + 12), c = ld4(ch + 16);
    a.z += t[0]; a.w += t[1]; b.x += t[2]; b.y += t[3]; b.z += t[4]; b.w += t[5]; c.x += t[6]; c.y += t[7];
    c.z += t[8]; c.w += t[9];
    st4(ch + 8, a);
    st4(ch + 12, b);
    st4(ch + 16, c);
}
template <int K> __device__ __forceinline__ void zero_arr(float (&x)[K]) {
#pragma unroll
    for (int q = 0; q < K; ++q) x[q] = 0.0f;
}

// pair index q in [0, 15) -> (s1 <= s2), lexicographic (the order of pair_le_index)
__device__ __forceinline__ void pair_of(int q, int &s1, int &s2) {
    s1 = 0;
    while (q >= NR - s1) {
        q -= NR - s1;
        ++s1;
    }
    s2 = s1 + q;
}

// position k of the item list (heaviest first) -> kind and run-time index
__device__ __forceinline__ void item_of(int k, int &kind, int &arg) {
    if (k == 0) { kind = IK_B; arg = 0; }
    else if (k <= 5) { kind = IK_E; arg = k - 1; }
    else if (k == 6) { kind = IK_B; arg = 1; }
    else if (k == 7) { kind = IK_F; arg = 0; }
    else if (k < 23) { kind = IK_D; arg = k - 8; }
    else if (k == 23) { kind = IK_B; arg = 2; }
    else if (k < 29) { kind = IK_C; arg = k - 24; }
    else { kind = IK_B; arg = k - 26; }          // 29 -> 3, 30 -> 4
}
// the r-th item of warp w of W (snake order: w, 2W-1-w, 2W+w, ...)
__device__ __forceinline__ int item_pos(int r, int w, int W) { return r * W + ((r & 1) ? W - 1 - w : w); }

// Item code is generic in the scalar T: float (features and dE/dPsi) or Dual (values with
// their tangents, for the parameter gradient).  Sources and sinks per lane:
//   MomSrc<T>  the atom's moments in the shared tile (Dual: moments and tangent moments)
//   GradIn<T>  dE/dG of the atom (Dual: two gradient rows, see k_contract_bwd_dual)
//   SlotAcc<T> the warp's slot row(s) for run-time gradient targets
template <typename T> struct MomSrc;
template <> struct MomSrc<float> {
    const float *r;
    __device__ __forceinline__ void v(int s, float (&x)[3]) const { ld_v(r + s * NC, x); }
    __device__ __forceinline__ void m(int s, float (&x)[6]) const { ld_m(r + s * NC, x); }
    __device__ __forceinline__ void t(int s, float (&x)[10]) const { ld_t(r + s * NC, x); }
    __device__ __forceinline__ float c0(int s) const { return r[s * NC]; }
};
template <> struct MomSrc<Dual> {
    const float *r, *d;
    template <int K>
    __device__ __forceinline__ static void zip(const float (&a)[K], const float (&b)[K], Dual (&x)[K]) {
#pragma unroll
        for (int q = 0; q < K; ++q) x[q] = {a[q], b[q]};
    }
    __device__ __forceinline__ void v(int s, Dual (&x)[3]) const {
        float a[3], b[3];
        ld_v(r + s * NC, a);
        ld_v(d + s * NC, b);
        zip(a, b, x);
    }
    __device__ __forceinline__ void m(int s, Dual (&x)[6]) const {
        float a[6], b[6];
        ld_m(r + s * NC, a);
        ld_m(d + s * NC, b);
        zip(a, b, x);
    }
    __device__ __forceinline__ void t(int s, Dual (&x)[10]) const {
        float a[10], b[10];
        ld_t(r + s * NC, a);
        ld_t(d + s * NC, b);
        zip(a, b, x);
    }
    __device__ __forceinline__ Dual c0(int s) const { return {r[s * NC], d[s * NC]}; }
};
template <typename T> struct GradIn;
template <> struct GradIn<float> {
    const float *g;
    __device__ __forceinline__ float operator()(int f) const { return g[f]; }
};
template <> struct GradIn<Dual> {
    const float *g, *gd;
    __device__ __forceinline__ Dual operator()(int f) const { return {g[f], gd[f]}; }
};
template <typename T> struct SlotAcc;
template <> struct SlotAcc<float> {
    float *a;
    __device__ __forceinline__ void v(int s, const float (&x)[3], float c0) const { add_v(a + s * NC, x, c0); }
    __device__ __forceinline__ void m(int s, const float (&x)[6]) const { add_m(a + s * NC, x); }
    __device__ __forceinline__ void t(int s, const float (&x)[10]) const { add_t(a + s * NC, x); }
};
template <> struct SlotAcc<Dual> {
    float *a, *ad;
    template <int K>
    __device__ __forceinline__ static void unzip(const Dual (&x)[K], float (&a)[K], float (&b)[K]) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            a[q] = x[q].v;
            b[q] = x[q].d;
        }
    }
    __device__ __forceinline__ void v(int s, const Dual (&x)[3], Dual c0) const {
        float p[3], q[3];
        unzip(x, p, q);
        add_v(a + s * NC, p, c0.v);
        add_v(ad + s * NC, q, c0.d);
    }
    __device__ __forceinline__ void m(int s, const Dual (&x)[6]) const {
        float p[6], q[6];
        unzip(x, p, q);
        add_m(a + s * NC, p);
        add_m(ad + s * NC, q);
    }
    __device__ __forceinline__ void t(int s, const Dual (&x)[10]) const {
        float p[10], q[10];
        unzip(x, p, q);
        add_t(a + s * NC, p);
        add_t(ad + s * NC, q);
    }
};
template <typename T, int K> __device__ __forceinline__ void zero_t(T (&x)[K]) {
#pragma unroll
    for (int q = 0; q < K; ++q) x[q] = zero<T>();
}

// register copy of an atom's vectors and matrices
template <typename T>
struct RegVM {
    T v[NR][3], m[NR][6];
};
template <typename T>
__device__ __forceinline__ void load_vm(const MomSrc<T> &src, RegVM<T> &p) {
#pragma unroll
    for (int s = 0; s < NR; ++s) {
        src.v(s, p.v[s]);
        src.m(s, p.m[s]);
    }
}

// Features of item (kind, arg) for this lane's atom (src = its moments) into out[0..360).
template <typename T>
__device__ __forceinline__ void fwd_item(int kind, int arg, const MomSrc<T> &src, const RegVM<T> &P,
                                         const FeatOut &out) {
    if (kind == IK_D) {                            // #7: Q_cd = T1_abc T2_abd, f = Q : M3;  #4: T1 : T2
        int s1, s2;
        pair_of(arg, s1, s2);
        T T1[10], T2[10];
        src.t(s1, T1);
        src.t(s2, T2);
        T f4 = zero<T>(), Q[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                T v = zero<T>();
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) v = mad(LT(T1, a, b, c), LT(T2, a, b, d), v);
                Q[c][d] = v;
                if (c == d) f4 += v;
            }
        out.put(FAM_OFF4 + arg, f4);
        const int f0 = FAM_OFF7 + f7_index(s1, s2, 0);
#pragma unroll
        for (int s3 = 0; s3 < NR; ++s3) {
            T f = zero<T>();
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int d = 0; d < 3; ++d) f = mad(Q[c][d], LM(P.m[s3], c, d), f);
            out.put(f0 + s3, f);
        }
    } else if (kind == IK_E) {                     // #8: U_a = T2_abc M3_bc, f = v1 . U
        const int t2 = arg;
        T T2[10];
        src.t(t2, T2);
#pragma unroll
        for (int s3 = 0; s3 < NR; ++s3) {
            T U[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                T v = zero<T>();
#pragma unroll
                for (int b = 0; b < 3; ++b)
#pragma unroll
                    for (int c = 0; c < 3; ++c) v = mad(LT(T2, a, b, c), LM(P.m[s3], b, c), v);
                U[a] = v;
            }
#pragma unroll
            for (int s1 = 0; s1 < NR; ++s1) {
                T f = zero<T>();
#pragma unroll
                for (int a = 0; a < 3; ++a) f = mad(P.v[s1][a], U[a], f);
                out.put(FAM_OFF8 + f8_index(s1, t2, s3), f);
            }
        }
    } else if (kind == IK_B) {                     // #5: tr(M1 M2 M3), s1 <= s2 <= s3
        const int s1 = arg;
        T M1[6];
        src.m(s1, M1);
#pragma unroll
        for (int s2 = 0; s2 < NR; ++s2) {
            if (s2 < s1) continue;
            T Nm[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    T v = zero<T>();
#pragma unroll
                    for (int b = 0; b < 3; ++b) v = mad(LM(M1, a, b), LM(P.m[s2], b, c), v);
                    Nm[a][c] = v;
                }
#pragma unroll
            for (int s3 = s2; s3 < NR; ++s3) {
                T f = zero<T>();
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int c = 0; c < 3; ++c) f = mad(Nm[a][c], LM(P.m[s3], c, a), f);
                out.put(FAM_OFF5 + f5_index(s1, s2, s3), f);
            }
        }
    } else if (kind == IK_C) {                     // #6: w = M2 v3, f = v1 . w, s1 <= s3
        const int t2 = arg;
        T M2[6];
        src.m(t2, M2);
#pragma unroll
        for (int s3 = 0; s3 < NR; ++s3) {
            T w[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                T v = zero<T>();
#pragma unroll
                for (int b = 0; b < 3; ++b) v = mad(LM(M2, a, b), P.v[s3][b], v);
                w[a] = v;
            }
#pragma unroll
            for (int s1 = 0; s1 <= s3; ++s1) {
                T f = zero<T>();
#pragma unroll
                for (int a = 0; a < 3; ++a) f = mad(P.v[s1][a], w[a], f);
                out.put(FAM_OFF6 + f6_index(s1, t2, s3), f);
            }
        }
    } else {                                       // #1, #2, #3
#pragma unroll
        for (int s = 0; s < NR; ++s) out.put(FAM_OFF1 + s, src.c0(s));
#pragma unroll
        for (int s1 = 0; s1 < NR; ++s1)
#pragma unroll
            for (int s2 = s1; s2 < NR; ++s2) {
                T f2 = zero<T>(), f3 = zero<T>();
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    f2 = mad(P.v[s1][a], P.v[s2][a], f2);
#pragma unroll
                    for (int b = 0; b < 3; ++b) f3 = mad(LM(P.m[s1], a, b), LM(P.m[s2], a, b), f3);
                }
                const int q = pair_le_index(s1, s2);
                out.put(FAM_OFF2 + q, f2);
                out.put(FAM_OFF3 + q, f3);
            }
    }
}

// register gradient accumulators of one atom: dE/dv_s, dE/dM_s, dE/dPsi0_s
template <typename T>
struct RegGrad {
    T v[NR][3], m[NR][6], c0[NR];
};

// dE/dPsi contributions of item (kind, arg) for this lane's atom (gb = its dE/dG): into
// the registers A, and into the slot row acc for the item's run-time tensor.  Full-tensor
// index loops write into unique accumulators, which sums all index permutations (the
// gradient with respect to the unique component).  Run-time targets that coincide
// (s1 == s2) are updated one after the other, so both contributions land.
template <typename T>
__device__ __forceinline__ void bwd_item(int kind, int arg, const MomSrc<T> &src, const RegVM<T> &P,
                                         const GradIn<T> &gb, RegGrad<T> &A, const SlotAcc<T> &acc) {
    if (kind == IK_D) {                            // #7 and #4
        int s1, s2;
        pair_of(arg, s1, s2);
        T T1[10], T2[10];
        src.t(s1, T1);
        src.t(s2, T2);
        const int f0 = FAM_OFF7 + f7_index(s1, s2, 0);
        const T g4 = gb(FAM_OFF4 + arg);
        T g[NR], Mw[6];                        // Mw = sum_s3 g M3 (symmetric)
        zero_t(Mw);
#pragma unroll
        for (int s3 = 0; s3 < NR; ++s3) {
            g[s3] = gb(f0 + s3);
#pragma unroll
            for (int u = 0; u < 6; ++u) Mw[u] = mad(g[s3], P.m[s3][u], Mw[u]);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int d = 0; d < 3; ++d) {          // Q_cd; d/dM3_cd = Q_cd
                T v = zero<T>();
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) v = mad(LT(T1, a, b, c), LT(T2, a, b, d), v);
#pragma unroll
                for (int s3 = 0; s3 < NR; ++s3) LM(A.m[s3], c, d) = mad(g[s3], v, LM(A.m[s3], c, d));
            }
        T t1[10], t2[10];                      // d/dT1_abc = g4 T2_abc + T2_abd Mw_cd, and T1 <-> T2
        zero_t(t1);
        zero_t(t2);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    T x1 = g4 * LT(T2, a, b, c), x2 = g4 * LT(T1, a, b, c);
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        x1 = mad(LT(T2, a, b, d), LM(Mw, c, d), x1);
                        x2 = mad(LT(T1, a, b, d), LM(Mw, d, c), x2);
                    }
                    LT(t1, a, b, c) += x1;
                    LT(t2, a, b, c) += x2;
                }
        acc.t(s1, t1);
        acc.t(s2, t2);
    } else if (kind == IK_E) {                     // #8
        const int t2 = arg;
        T T2[10], at[10];
        src.t(t2, T2);
        zero_t(at);
#pragma unroll
        for (int s3 = 0; s3 < NR; ++s3) {
            T U[3], Vw[3];
            zero_t(Vw);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                T v = zero<T>();
#pragma unroll
                for (int b = 0; b < 3; ++b)
#pragma unroll
                    for (int c = 0; c < 3; ++c) v = mad(LT(T2, a, b, c), LM(P.m[s3], b, c), v);
                U[a] = v;
            }
#pragma unroll
            for (int s1 = 0; s1 < NR; ++s1) {      // d/dv1 = g U; Vw = sum_s1 g v1
                const T g = gb(FAM_OFF8 + f8_index(s1, t2, s3));
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    A.v[s1][a] = mad(g, U[a], A.v[s1][a]);
                    Vw[a] = mad(g, P.v[s1][a], Vw[a]);
                }
            }
#pragma unroll
            for (int a = 0; a < 3; ++a)            // d/dT2_abc = Vw_a M3_bc, d/dM3_bc = Vw_a T2_abc
#pragma unroll
                for (int b = 0; b < 3; ++b)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        LT(at, a, b, c) = mad(Vw[a], LM(P.m[s3], b, c), LT(at, a, b, c));
                        LM(A.m[s3], b, c) = mad(Vw[a], LT(T2, a, b, c), LM(A.m[s3], b, c));
                    }
        }
        acc.t(t2, at);
    } else if (kind == IK_B) {                     // #5: s1 <= s2 <= s3
        const int s1 = arg;
        T M1[6], a1[6];
        src.m(s1, M1);
        zero_t(a1);
#pragma unroll
        for (int s2 = 0; s2 < NR; ++s2) {
            if (s2 < s1) continue;
            T Nm[3][3], Mg[6];                 // Nm = M1 M2, Mg = sum_s3 g M3
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    T v = zero<T>();
#pragma unroll
                    for (int b = 0; b < 3; ++b) v = mad(LM(M1, a, b), LM(P.m[s2], b, c), v);
                    Nm[a][c] = v;
                }
            zero_t(Mg);
#pragma unroll
            for (int s3 = s2; s3 < NR; ++s3) {     // d/d(M3)_ba = (M1 M2)_ab
                const T g = gb(FAM_OFF5 + f5_index(s1, s2, s3));
#pragma unroll
                for (int u = 0; u < 6; ++u) Mg[u] = mad(g, P.m[s3][u], Mg[u]);
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) LM(A.m[s3], b, a) = mad(g, Nm[a][b], LM(A.m[s3], b, a));
            }
#pragma unroll
            for (int a = 0; a < 3; ++a)            // d/d(M1)_ba = (M2 Mg)_ab, d/d(M2)_ba = (Mg M1)_ab
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    T x1 = zero<T>(), x2 = zero<T>();
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        x1 = mad(LM(P.m[s2], a, c), LM(Mg, c, b), x1);
                        x2 = mad(LM(Mg, a, c), LM(M1, c, b), x2);
                    }
                    LM(a1, b, a) += x1;
                    LM(A.m[s2], b, a) += x2;
                }
        }
        acc.m(s1, a1);
    } else if (kind == IK_C) {                     // #6: s1 <= s3
        const int t2 = arg;
        T M2[6], am[6];
        src.m(t2, M2);
        zero_t(am);
#pragma unroll
        for (int s3 = 0; s3 < NR; ++s3) {
            T w[3], vg[3];
            zero_t(vg);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                T v = zero<T>();
#pragma unroll
                for (int b = 0; b < 3; ++b) v = mad(LM(M2, a, b), P.v[s3][b], v);
                w[a] = v;
            }
#pragma unroll
            for (int s1 = 0; s1 <= s3; ++s1) {     // d/dv1 = g M2 v3; vg = sum_s1 g v1
                const T g = gb(FAM_OFF6 + f6_index(s1, t2, s3));
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    A.v[s1][a] = mad(g, w[a], A.v[s1][a]);
                    vg[a] = mad(g, P.v[s1][a], vg[a]);
                }
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) {          // d/dM2_ab = vg_a v3_b, d/dv3 = M2 vg
                T v = zero<T>();
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    LM(am, a, b) = mad(vg[a], P.v[s3][b], LM(am, a, b));
                    v = mad(LM(M2, a, b), vg[b], v);
                }
                A.v[s3][a] += v;
            }
        }
        acc.m(t2, am);
    } else {                                       // #1, #2, #3
#pragma unroll
        for (int s = 0; s < NR; ++s) A.c0[s] += gb(FAM_OFF1 + s);
#pragma unroll
        for (int s1 = 0; s1 < NR; ++s1)
#pragma unroll
            for (int s2 = s1; s2 < NR; ++s2) {
                const int q = pair_le_index(s1, s2);
                const T g2 = gb(FAM_OFF2 + q), g3 = gb(FAM_OFF3 + q);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    A.v[s1][a] = mad(g2, P.v[s2][a], A.v[s1][a]);
                    A.v[s2][a] = mad(g2, P.v[s1][a], A.v[s2][a]);
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        LM(A.m[s1], a, b) = mad(g3, LM(P.m[s2], a, b), LM(A.m[s1], a, b));
                        LM(A.m[s2], a, b) = mad(g3, LM(P.m[s1], a, b), LM(A.m[s2], a, b));
                    }
                }
            }
    }
}

// psi rows m0..m0+31 (zero past N) into the shared tile [32][100]
template <int NT>
__device__ __forceinline__ void stage_psi(const float *__restrict__ psi, int m0, int N, float *ptile) {
    constexpr int V4 = NPSI / 4;
    const float4 *src = reinterpret_cast<const float4 *>(psi + (size_t)m0 * NPSI);
    float4 *dst = reinterpret_cast<float4 *>(ptile);
    for (int idx = threadIdx.x; idx < CT_ATOMS * V4; idx += NT)
        dst[idx] = m0 + idx / V4 < N ? __ldg(src + idx) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

template <typename OutT, int W>
__global__ void __launch_bounds__(W * 32) k_contract_fwd(const float *__restrict__ psi, int N, int Mp,
                                                         OutT *__restrict__ G, float *__restrict__ G32, int lo_out) {
    extern __shared__ __align__(16) float smf[];
    float *ptile = smf;                            // [32][100]
    float *tile = smf + CT_ATOMS * NPSI;           // [32][GT_STRIDE] features
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * CT_ATOMS;
    griddep_wait();
    stage_psi<W * 32>(psi, m0, N, ptile);
    __syncthreads();
    const MomSrc<float> src{ptile + lane * NPSI};
    const FeatOut out{tile + lane * GT_STRIDE, nullptr};
    RegVM<float> P;
    load_vm(src, P);
    for (int r = 0;; ++r) {
        const int k = item_pos(r, warp, W);
        if (k >= IT_COUNT) break;
        int kind, arg;
        item_of(k, kind, arg);
        fwd_item(kind, arg, src, P, out);
    }
    __syncthreads();
    // 16-byte stores of 8 columns (BF16: a hi/lo row pair [hi(384) | lo(384)]) or 4 columns.
    // A warp takes 8 rows x 4 column groups: with the odd row stride the scalar tile reads
    // are free of bank conflicts, and each row gets 64 contiguous bytes.
    constexpr int CW = sizeof(OutT) == 2 ? 8 : 4, NCW = NFP / CW;
    static_assert(NCW % 4 == 0, "column groups per row");
    for (int idx = threadIdx.x; idx < CT_ATOMS * NCW; idx += W * 32) {
        const int chunk = idx >> 5, l = idx & 31;
        const int r = 8 * (chunk & 3) + (l >> 2), c = 4 * (chunk >> 2) + (l & 3), m = m0 + r;
        if (m >= Mp) continue;
        float v[CW];
#pragma unroll
        for (int j = 0; j < CW; ++j) v[j] = c * CW + j < NF ? tile[r * GT_STRIDE + c * CW + j] : 0.0f;
        if constexpr (sizeof(OutT) == 2) {
            __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                hi[j] = __float2bfloat16_rn(v[j]);
                lo[j] = __float2bfloat16_rn(v[j] - __bfloat162float(hi[j]));
            }
            __nv_bfloat16 *orow = reinterpret_cast<__nv_bfloat16 *>(G) + (size_t)m * 2 * NFP + c * 8;
            *reinterpret_cast<uint4 *>(orow) = *reinterpret_cast<const uint4 *>(hi);
            if (lo_out) *reinterpret_cast<uint4 *>(orow + NFP) = *reinterpret_cast<const uint4 *>(lo);
        } else {
            *reinterpret_cast<float4 *>(G + (size_t)m * NFP + c * 4) = make_float4(v[0], v[1], v[2], v[3]);
        }
    }
    if (G32 != nullptr) {
        for (int idx = threadIdx.x; idx < CT_ATOMS * NF; idx += W * 32) {
            const int r = idx / NF, f = idx - r * NF, m = m0 + r;
            if (m < N) G32[(size_t)m * NF + f] = tile[r * GT_STRIDE + f];
        }
    }
}

template <int W>
// Shallow-ensemble heads in one launch: bph blocks per head, block b taking head b / bph with
// its dE/dG at dG + head dg_hs and its dE/dPsi at dpsi + head dpsi_hs (one head: bph = grid)
__global__ void __launch_bounds__(W * 32) k_contract_bwd(const float *__restrict__ psi, const float *__restrict__ dG,
                                                         int N, float *__restrict__ dpsi, int dg_tiled, int bph,
                                                         size_t dg_hs, size_t dpsi_hs) {
    extern __shared__ __align__(16) float smb[];
    float *ptile = smb;                                    // [32][100] moments
    float *slots = ptile + CT_ATOMS * NPSI;                // W x [32][100] partial dE/dPsi
    float *gtile = slots + W * CT_ATOMS * NPSI;            // [32][GT_STRIDE] dE/dG
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int head = blockIdx.x / bph;
    const int m0 = (blockIdx.x - head * bph) * CT_ATOMS;
    dG += head * dg_hs;
    dpsi += head * dpsi_hs;
    griddep_wait();
    stage_psi<W * 32>(psi, m0, N, ptile);
    {
        float4 *mine = reinterpret_cast<float4 *>(slots + warp * CT_ATOMS * NPSI);
        for (int q = lane; q < CT_ATOMS * NPSI / 4; q += 32) mine[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    stage_rows<W * 32>(dG, m0, N, gtile, dg_tiled != 0);    // ends with __syncthreads()
    const MomSrc<float> src{ptile + lane * NPSI};
    const GradIn<float> gb{gtile + lane * GT_STRIDE};
    const SlotAcc<float> acc{slots + warp * CT_ATOMS * NPSI + lane * NPSI};
    RegVM<float> P;
    load_vm(src, P);
    RegGrad<float> A;
#pragma unroll
    for (int s = 0; s < NR; ++s) {
        zero_t(A.v[s]);
        zero_t(A.m[s]);
        A.c0[s] = 0.0f;
    }
    for (int r = 0;; ++r) {
        const int k = item_pos(r, warp, W);
        if (k >= IT_COUNT) break;
        int kind, arg;
        item_of(k, kind, arg);
        bwd_item(kind, arg, src, P, gb, A, acc);
    }
#pragma unroll
    for (int s = 0; s < NR; ++s) {
        acc.v(s, A.v[s], A.c0[s]);
        acc.m(s, A.m[s]);
    }
    __syncthreads();
    const float4 *s4 = reinterpret_cast<const float4 *>(slots);
    constexpr int V4 = NPSI / 4, SLOT4 = CT_ATOMS * V4;
    float4 *d4 = reinterpret_cast<float4 *>(dpsi + (size_t)m0 * NPSI);
    for (int idx = threadIdx.x; idx < SLOT4; idx += W * 32) {
        if (m0 + idx / V4 >= N) break;
        float4 v = s4[idx];
#pragma unroll
        for (int w = 1; w < W; ++w) {
            const float4 x = s4[w * SLOT4 + idx];
            v.x += x.x; v.y += x.y; v.z += x.z; v.w += x.w;
        }
        d4[idx] = v;
    }
}

// ------------------------------------------------------------------ parameter-gradient variants
// The same work items on dual numbers (value, tangent along Psid).
//
// Forward: features G and their tangents Gd = dG/dPsi . Psid, written as the stacked GEMM
// operand GG [2 Mp][384] (rows m: G, rows Mp + m: Gd; FP32).
template <int W>
__global__ void __launch_bounds__(W * 32) k_contract_fwd_dual(const float *__restrict__ psi,
                                                              const float *__restrict__ psid, int N, int Mp,
                                                              float *__restrict__ GG) {
    extern __shared__ __align__(16) float smd[];
    float *ptile = smd, *pdtile = smd + CT_ATOMS * NPSI;          // [32][100] each
    float *tv = pdtile + CT_ATOMS * NPSI, *td = tv + CT_ATOMS * GT_STRIDE;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * CT_ATOMS;
    griddep_wait();
    stage_psi<W * 32>(psi, m0, N, ptile);
    stage_psi<W * 32>(psid, m0, N, pdtile);
    __syncthreads();
    const MomSrc<Dual> src{ptile + lane * NPSI, pdtile + lane * NPSI};
    const FeatOut out{tv + lane * GT_STRIDE, td + lane * GT_STRIDE};
    RegVM<Dual> P;
    load_vm(src, P);
    for (int r = 0;; ++r) {
        const int k = item_pos(r, warp, W);
        if (k >= IT_COUNT) break;
        int kind, arg;
        item_of(k, kind, arg);
        fwd_item(kind, arg, src, P, out);
    }
    __syncthreads();
    constexpr int NCW = NFP / 4;                                  // 8 rows x 4 column groups per warp
    for (int idx = threadIdx.x; idx < CT_ATOMS * NCW; idx += W * 32) {
        const int chunk = idx >> 5, l = idx & 31;
        const int r = 8 * (chunk & 3) + (l >> 2), c = 4 * (chunk >> 2) + (l & 3), m = m0 + r;
        if (m >= Mp) continue;
        float v[4], d[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool in = c * 4 + j < NF;
            v[j] = in ? tv[r * GT_STRIDE + c * 4 + j] : 0.0f;
            d[j] = in ? td[r * GT_STRIDE + c * 4 + j] : 0.0f;
        }
        *reinterpret_cast<float4 *>(GG + (size_t)m * NFP + c * 4) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4 *>(GG + (size_t)(Mp + m) * NFP + c * 4) = make_float4(d[0], d[1], d[2], d[3]);
    }
}

// Backward.  With Gb = dJ/dG and Gdb = dJ/dGd (stacked in Gbs [2 Mp][384]) the moment
// adjoints are
//   psidb = J^T Gdb,   psib = J^T Gb + (dJ^T/dPsi . Psid) Gdb,   J = dG/dPsi.
// J^T g is linear in g, so one evaluation of the backward items on duals with moments
// Psi + e Psid and gradient rows Gdb + e Gb gives psidb as the value and psib as the
// tangent.  Each warp has a value slot and a tangent slot; the slots are summed in warp
// order (deterministic).
template <int W>
__global__ void __launch_bounds__(W * 32) k_contract_bwd_dual(const float *__restrict__ psi,
                                                              const float *__restrict__ psid,
                                                              const float *__restrict__ Gbs, int N, int Mp,
                                                              float *__restrict__ psib, float *__restrict__ psidb) {
    extern __shared__ __align__(16) float smd[];
    float *ptile = smd, *pdtile = smd + CT_ATOMS * NPSI;          // [32][100] each
    float *slots = pdtile + CT_ATOMS * NPSI;                      // W x (value, tangent) x [32][100]
    float *gtile = slots + 2 * W * CT_ATOMS * NPSI;               // Gb rows [32][GT_STRIDE]
    float *gdtile = gtile + CT_ATOMS * GT_STRIDE;                 // Gdb rows
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * CT_ATOMS;
    griddep_wait();
    stage_psi<W * 32>(psi, m0, N, ptile);
    stage_psi<W * 32>(psid, m0, N, pdtile);
    {
        float4 *mine = reinterpret_cast<float4 *>(slots + 2 * warp * CT_ATOMS * NPSI);
        for (int q = lane; q < 2 * CT_ATOMS * NPSI / 4; q += 32) mine[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    stage_rows<W * 32>(Gbs, m0, N, gtile);                        // each ends with __syncthreads()
    stage_rows<W * 32>(Gbs + (size_t)Mp * NFP, m0, N, gdtile);
    const MomSrc<Dual> src{ptile + lane * NPSI, pdtile + lane * NPSI};
    const GradIn<Dual> gb{gdtile + lane * GT_STRIDE, gtile + lane * GT_STRIDE};
    float *mine = slots + 2 * warp * CT_ATOMS * NPSI;
    const SlotAcc<Dual> acc{mine + lane * NPSI, mine + CT_ATOMS * NPSI + lane * NPSI};
    RegVM<Dual> P;
    load_vm(src, P);
    RegGrad<Dual> A;
#pragma unroll
    for (int s = 0; s < NR; ++s) {
        zero_t(A.v[s]);
        zero_t(A.m[s]);
        A.c0[s] = zero<Dual>();
    }
    for (int r = 0;; ++r) {
        const int k = item_pos(r, warp, W);
        if (k >= IT_COUNT) break;
        int kind, arg;
        item_of(k, kind, arg);
        bwd_item(kind, arg, src, P, gb, A, acc);
    }
#pragma unroll
    for (int s = 0; s < NR; ++s) {
        acc.v(s, A.v[s], A.c0[s]);
        acc.m(s, A.m[s]);
    }
    __syncthreads();
    const float4 *s4 = reinterpret_cast<const float4 *>(slots);
    constexpr int V4 = NPSI / 4, SLOT4 = CT_ATOMS * V4;
    float4 *dv = reinterpret_cast<float4 *>(psidb + (size_t)m0 * NPSI);
    float4 *dd = reinterpret_cast<float4 *>(psib + (size_t)m0 * NPSI);
    for (int idx = threadIdx.x; idx < SLOT4; idx += W * 32) {
        if (m0 + idx / V4 >= N) break;
        float4 v = s4[idx], d = s4[SLOT4 + idx];
#pragma unroll
        for (int w = 1; w < W; ++w) {
            const float4 x = s4[2 * w * SLOT4 + idx], y = s4[(2 * w + 1) * SLOT4 + idx];
            v.x += x.x; v.y += x.y; v.z += x.z; v.w += x.w;
            d.x += y.x; d.y += y.y; d.z += y.z; d.w += y.w;
        }
        dv[idx] = v;
        dd[idx] = d;
    }
}

// ------------------------------------------------------------------ launchers
// Warps per block of the dual kernels: the forward stages 118 KB (moments, tangents and two
// feature tiles) with 8 warps; the backward 220 KB (two moment tiles, two gradient tiles and
// value/tangent slots for 4 warps).
constexpr int CT_FWD_DUAL_W = 8, CT_BWD_DUAL_W = 4;
constexpr size_t ct_fwd_dual_smem() { return sizeof(float) * (2 * CT_ATOMS * NPSI + 2 * CT_ATOMS * GT_STRIDE); }
constexpr size_t ct_bwd_dual_smem() {
    return sizeof(float) * ((2 + 2 * CT_BWD_DUAL_W) * CT_ATOMS * NPSI + 2 * CT_ATOMS * GT_STRIDE);
}
static_assert(ct_fwd_dual_smem() <= 227 * 1024 && ct_bwd_dual_smem() <= 227 * 1024,
              "dual contraction tiles exceed the shared memory of a block");

void launch_contract_fwd_dual(const float *psi, const float *psid, int N, int Mp, float *GG, cudaStream_t st) {
    const int blocks = (Mp + CT_ATOMS - 1) / CT_ATOMS;
    static PerDeviceOnce attr;
    if (attr.first()) {
        cudaFuncSetAttribute(k_contract_fwd_dual<CT_FWD_DUAL_W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ct_fwd_dual_smem());
    }
    if (blocks > 0) {
        launch_pdl(k_contract_fwd_dual<CT_FWD_DUAL_W>, dim3(blocks), dim3(CT_FWD_DUAL_W * 32), ct_fwd_dual_smem(), st,
                   psi, psid, N, Mp, GG);
        note_launches(1);
    }
}

void launch_contract_bwd_dual(const float *psi, const float *psid, const float *Gbs, int N, int Mp, float *psib,
                              float *psidb, cudaStream_t st) {
    const int blocks = (N + CT_ATOMS - 1) / CT_ATOMS;
    static PerDeviceOnce attr;
    if (attr.first()) {
        cudaFuncSetAttribute(k_contract_bwd_dual<CT_BWD_DUAL_W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ct_bwd_dual_smem());
    }
    if (blocks > 0) {
        launch_pdl(k_contract_bwd_dual<CT_BWD_DUAL_W>, dim3(blocks), dim3(CT_BWD_DUAL_W * 32), ct_bwd_dual_smem(), st,
                   psi, psid, Gbs, N, Mp, psib, psidb);
        note_launches(1);
    }
}

// Warps per block of the item kernels.  The forward uses 8 (its 59 KB of shared memory let
// three blocks share an SM); the backward uses 4 (110 KB with the four private slots, two
// blocks per SM).  A grid of fewer blocks than SMs (systems under 32 x #SMs atoms) leaves
// SMs idle, so there the 31 items of a block are shared by twice the warps instead: 16 in
// the forward (same shared memory, 128 registers), 8 in the backward (161 KB, one block per
// SM).  The forward's features do not depend on the split; the backward sums its warps'
// slots in warp order, so its last bits depend on the warp count (fixed for a given size).
constexpr int CT_FWD_W = 8, CT_BWD_W = 4;
constexpr size_t ct_fwd_smem() { return sizeof(float) * (CT_ATOMS * NPSI + CT_ATOMS * GT_STRIDE); }
template <int W> constexpr size_t ct_bwd_smem() {
    return sizeof(float) * ((W + 1) * CT_ATOMS * NPSI + CT_ATOMS * GT_STRIDE);
}
static_assert(ct_bwd_smem<2 * CT_BWD_W>() <= 227 * 1024, "backward with doubled warps fits in shared memory");

int device_sm_count() {
    static int cnt[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    int &c = cnt[dev & 63];
    if (c <= 0) cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    return c > 0 ? c : 1;
}

template <typename OutT, int W>
static void launch_fwd_w(int blocks, const float *psi, int N, int Mp, OutT *G, float *features_out, int lo_out,
                         cudaStream_t st) {
    static PerDeviceOnce attr;
    if (attr.first()) {
        cudaFuncSetAttribute(k_contract_fwd<OutT, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ct_fwd_smem());
    }
    launch_pdl(k_contract_fwd<OutT, W>, dim3(blocks), dim3(W * 32), ct_fwd_smem(), st, psi, N, Mp, G, features_out,
               lo_out);
    note_launches(1);
}

template <typename OutT>
static void launch_fwd_items(const float *psi, int N, int Mp, OutT *G, float *features_out, int lo_out,
                             cudaStream_t st) {
    const int blocks = (Mp + CT_ATOMS - 1) / CT_ATOMS;
    if (blocks <= 0) return;
    if (blocks < device_sm_count())
        launch_fwd_w<OutT, 2 * CT_FWD_W>(blocks, psi, N, Mp, G, features_out, lo_out, st);
    else
        launch_fwd_w<OutT, CT_FWD_W>(blocks, psi, N, Mp, G, features_out, lo_out, st);
}

void launch_contract_fwd_f32(const float *psi, int N, int Mp, float *G, float *features_out, cudaStream_t st) {
    launch_fwd_items<float>(psi, N, Mp, G, features_out, 0, st);
}

void launch_contract_fwd_bf16(const float *psi, int N, int Mp, __nv_bfloat16 *G, float *features_out, bool lo_out,
                              cudaStream_t st) {
    launch_fwd_items<__nv_bfloat16>(psi, N, Mp, G, features_out, lo_out ? 1 : 0, st);
}

template <int W>
static void launch_bwd_w(int blocks, const float *psi, const float *dG, int N, float *dpsi, int dg_tiled, int bph,
                         size_t dg_hs, size_t dpsi_hs, cudaStream_t st) {
    static PerDeviceOnce attr;
    if (attr.first()) {
        cudaFuncSetAttribute(k_contract_bwd<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ct_bwd_smem<W>());
    }
    launch_pdl(k_contract_bwd<W>, dim3(blocks), dim3(W * 32), ct_bwd_smem<W>(), st, psi, dG, N, dpsi, dg_tiled, bph,
               dg_hs, dpsi_hs);
    note_launches(1);
}

void launch_contract_bwd(const float *psi, const float *dG, int N, float *dpsi, cudaStream_t st, bool dg_tiled,
                         int heads, size_t dg_head_stride) {
    const int bph = (N + CT_ATOMS - 1) / CT_ATOMS;
    if (bph <= 0 || heads < 1) return;
    const int blocks = bph * heads;
    const size_t dpsi_hs = (size_t)N * NPSI;
    if (blocks < device_sm_count())
        launch_bwd_w<2 * CT_BWD_W>(blocks, psi, dG, N, dpsi, dg_tiled ? 1 : 0, bph, dg_head_stride, dpsi_hs, st);
    else
        launch_bwd_w<CT_BWD_W>(blocks, psi, dG, N, dpsi, dg_tiled ? 1 : 0, bph, dg_head_stride, dpsi_hs, st);
}

}  // namespace gm
