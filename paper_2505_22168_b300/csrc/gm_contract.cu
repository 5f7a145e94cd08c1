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
// Layout: a block holds 32 atoms (one per lane) and 8 warps; warp w evaluates feature
// group w for all 32 atoms, so every warp runs one code path.  The forward and backward
// kernels are capped at 128 registers so that two blocks share an SM: the latency-bound
// group code gains more from the second block than it loses to the few spills (measured on
// B300 at 16,384 atoms: backward 105 -> 63 us, forward 39 -> 28 us; three blocks spill too
// much).  Groups: 0 = #1-#4,
// 1 = #5, 2 = #6, 3-5 = #7 split by s1 ({0}, {1,4}, {2,3}), 6-7 = #8 split by s2
// ({0,1}, {2,3,4}).  The 360 features of the 32 atoms are staged in shared memory and
// written as coalesced rows of the [M][384] GEMM operand (columns 360..383 are zero).
//
// Backward: each group accumulates its contribution to dE/dPsi (unique components, 100
// per atom) in registers, using full-tensor index loops whose writes land in the unique
// accumulators (this sums all index permutations, i.e. the gradient with respect to
// the unique component); the 8 partial gradients are added in a fixed group order.
#include "gm_contract.h"

namespace gm {

constexpr int CT_ATOMS = 32;
constexpr int CT_THREADS = 256;
constexpr int GT_STRIDE = NF + 1;
constexpr int AC_STRIDE = NPSI + 1;

#define PV(s, a) P[(s) * NC + idx1(a)]
#define PM(s, a, b) P[(s) * NC + idx2(a, b)]
#define PT(s, a, b, c) P[(s) * NC + idx3(a, b, c)]
#define AV(s, a) A[(s) * NC + idx1(a)]
#define AM(s, a, b) A[(s) * NC + idx2(a, b)]
#define AT(s, a, b, c) A[(s) * NC + idx3(a, b, c)]

// Forward-mode dual number (value, derivative along a tangent direction).  The features
// are polynomials of the moments, so running the same group code on duals gives exact
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

__host__ __device__ constexpr bool f7_group_has(int part, int s1) {
    return part == 3 ? s1 == 0 : (part == 4 ? (s1 == 1 || s1 == 4) : (s1 == 2 || s1 == 3));
}
__host__ __device__ constexpr bool f8_group_has(int part, int s2) { return part == 6 ? s2 <= 1 : s2 >= 2; }

__device__ __forceinline__ void load_psi(const float *__restrict__ psi, int m, int N, float (&P)[NPSI]) {
    if (m < N) {
        const float4 *p4 = reinterpret_cast<const float4 *>(psi + (size_t)m * NPSI);
#pragma unroll
        for (int q = 0; q < NPSI / 4; ++q) {
            const float4 v = p4[q];
            P[4 * q] = v.x; P[4 * q + 1] = v.y; P[4 * q + 2] = v.z; P[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < NPSI; ++q) P[q] = 0.0f;
    }
}

// ------------------------------------------------------------------ forward groups
template <int PART, typename T>
__device__ __forceinline__ void fwd_group(const T (&P)[NPSI], const FeatOut &gt) {
    if (PART == 0) {
#pragma unroll
        for (int s = 0; s < NR; ++s) gt.put(FAM_OFF1 + s, P[s * NC]);
#pragma unroll
        for (int s1 = 0; s1 < NR; ++s1)
#pragma unroll
            for (int s2 = s1; s2 < NR; ++s2) {
                T f2 = zero<T>(), f3 = zero<T>(), f4 = zero<T>();
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    f2 = mad(PV(s1, a), PV(s2, a), f2);
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        f3 = mad(PM(s1, a, b), PM(s2, a, b), f3);
#pragma unroll
                        for (int c = 0; c < 3; ++c) f4 = mad(PT(s1, a, b, c), PT(s2, a, b, c), f4);
                    }
                }
                const int q = pair_le_index(s1, s2);
                gt.put(FAM_OFF2 + q, f2);
                gt.put(FAM_OFF3 + q, f3);
                gt.put(FAM_OFF4 + q, f4);
            }
    } else if (PART == 1) {
        // fixed trip counts with guards: triangular bounds left the loops rolled and the
        // moments in local memory
#pragma unroll
        for (int s1 = 0; s1 < NR; ++s1)
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
                        for (int b = 0; b < 3; ++b) v = mad(PM(s1, a, b), PM(s2, b, c), v);
                        Nm[a][c] = v;
                    }
#pragma unroll
                for (int s3 = 0; s3 < NR; ++s3) {
                    if (s3 < s2) continue;
                    T f = zero<T>();
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int c = 0; c < 3; ++c) f = mad(Nm[a][c], PM(s3, c, a), f);
                    gt.put(FAM_OFF5 + f5_index(s1, s2, s3), f);
                }
            }
    } else if (PART == 2) {
#pragma unroll
        for (int s2 = 0; s2 < NR; ++s2)
#pragma unroll
            for (int s3 = 0; s3 < NR; ++s3) {
                T w[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    T v = zero<T>();
#pragma unroll
                    for (int b = 0; b < 3; ++b) v = mad(PM(s2, a, b), PV(s3, b), v);
                    w[a] = v;
                }
#pragma unroll
                for (int s1 = 0; s1 <= s3; ++s1) {
                    T f = zero<T>();
#pragma unroll
                    for (int a = 0; a < 3; ++a) f = mad(PV(s1, a), w[a], f);
                    gt.put(FAM_OFF6 + f6_index(s1, s2, s3), f);
                }
            }
    } else if (PART >= 3 && PART <= 5) {
#pragma unroll
        for (int s1 = 0; s1 < NR; ++s1) {
            if (!f7_group_has(PART, s1)) continue;
#pragma unroll
            for (int s2 = s1; s2 < NR; ++s2) {
                T Q[3][3];
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        T v = zero<T>();
#pragma unroll
                        for (int a = 0; a < 3; ++a)
#pragma unroll
                            for (int b = 0; b < 3; ++b) v = mad(PT(s1, a, b, c), PT(s2, a, b, d), v);
                        Q[c][d] = v;
                    }
#pragma unroll
                for (int s3 = 0; s3 < NR; ++s3) {
                    T f = zero<T>();
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int d = 0; d < 3; ++d) f = mad(Q[c][d], PM(s3, c, d), f);
                    gt.put(FAM_OFF7 + f7_index(s1, s2, s3), f);
                }
            }
        }
    } else {
#pragma unroll
        for (int s2 = 0; s2 < NR; ++s2) {
            if (!f8_group_has(PART, s2)) continue;
#pragma unroll
            for (int s3 = 0; s3 < NR; ++s3) {
                T U[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    T v = zero<T>();
#pragma unroll
                    for (int b = 0; b < 3; ++b)
#pragma unroll
                        for (int c = 0; c < 3; ++c) v = mad(PT(s2, a, b, c), PM(s3, b, c), v);
                    U[a] = v;
                }
#pragma unroll
                for (int s1 = 0; s1 < NR; ++s1) {
                    T f = zero<T>();
#pragma unroll
                    for (int a = 0; a < 3; ++a) f = mad(PV(s1, a), U[a], f);
                    gt.put(FAM_OFF8 + f8_index(s1, s2, s3), f);
                }
            }
        }
    }
}

template <typename OutT>
__global__ void __launch_bounds__(CT_THREADS, 2) k_contract_fwd(const float *__restrict__ psi, int N, int Mp,
                                                                OutT *__restrict__ G, float *__restrict__ G32,
                                                                int lo_out) {
    extern __shared__ float tile[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * CT_ATOMS;
    float P[NPSI];
    load_psi(psi, m0 + lane, N, P);
    const FeatOut gt{tile + lane * GT_STRIDE, nullptr};
    switch (warp) {
    case 0: fwd_group<0>(P, gt); break;
    case 1: fwd_group<1>(P, gt); break;
    case 2: fwd_group<2>(P, gt); break;
    case 3: fwd_group<3>(P, gt); break;
    case 4: fwd_group<4>(P, gt); break;
    case 5: fwd_group<5>(P, gt); break;
    case 6: fwd_group<6>(P, gt); break;
    default: fwd_group<7>(P, gt); break;
    }
    __syncthreads();
    // 16-byte stores of 8 columns (BF16: a hi/lo row pair [hi(384) | lo(384)]) or 4 columns
    constexpr int CW = sizeof(OutT) == 2 ? 8 : 4, NCW = NFP / CW;
    for (int idx = threadIdx.x; idx < CT_ATOMS * NCW; idx += CT_THREADS) {
        const int r = idx / NCW, c = idx - r * NCW, m = m0 + r;
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
            __nv_bfloat16 *row = reinterpret_cast<__nv_bfloat16 *>(G) + (size_t)m * 2 * NFP + c * 8;
            *reinterpret_cast<uint4 *>(row) = *reinterpret_cast<const uint4 *>(hi);
            if (lo_out) *reinterpret_cast<uint4 *>(row + NFP) = *reinterpret_cast<const uint4 *>(lo);
        } else {
            *reinterpret_cast<float4 *>(G + (size_t)m * NFP + c * 4) = make_float4(v[0], v[1], v[2], v[3]);
        }
    }
    if (G32 != nullptr) {
        for (int idx = threadIdx.x; idx < CT_ATOMS * NF; idx += CT_THREADS) {
            const int r = idx / NF, f = idx - r * NF, m = m0 + r;
            if (m < N) G32[(size_t)m * NF + f] = tile[r * GT_STRIDE + f];
        }
    }
}

// ------------------------------------------------------------------ backward groups
// Backward units: FAM 0 = families #1-#4; FAM 5, 6, 7, 8 = that family restricted by MASK
// (a bit set per radial index: s1 for #5 and #7, s2 for #6 and #8).
template <int FAM, int MASK, typename T>
__device__ __forceinline__ void bwd_unit(const T (&P)[NPSI], const float *gb, T (&A)[NPSI]) {
    if (FAM == 0) {
#pragma unroll
        for (int s = 0; s < NR; ++s) A[s * NC] += gb[FAM_OFF1 + s];
#pragma unroll
        for (int s1 = 0; s1 < NR; ++s1)
#pragma unroll
            for (int s2 = s1; s2 < NR; ++s2) {
                const int q = pair_le_index(s1, s2);
                const float g2 = gb[FAM_OFF2 + q], g3 = gb[FAM_OFF3 + q], g4 = gb[FAM_OFF4 + q];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    AV(s1, a) = mad(g2, PV(s2, a), AV(s1, a));
                    AV(s2, a) = mad(g2, PV(s1, a), AV(s2, a));
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        AM(s1, a, b) = mad(g3, PM(s2, a, b), AM(s1, a, b));
                        AM(s2, a, b) = mad(g3, PM(s1, a, b), AM(s2, a, b));
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            AT(s1, a, b, c) = mad(g4, PT(s2, a, b, c), AT(s1, a, b, c));
                            AT(s2, a, b, c) = mad(g4, PT(s1, a, b, c), AT(s2, a, b, c));
                        }
                    }
                }
            }
    } else if (FAM == 5) {
#pragma unroll
        for (int s1 = 0; s1 < NR; ++s1)
#pragma unroll
            for (int s2 = s1; s2 < NR; ++s2)
                if ((MASK >> s1) & 1)
#pragma unroll
                for (int s3 = s2; s3 < NR; ++s3) {
                    const float g = gb[FAM_OFF5 + f5_index(s1, s2, s3)];
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int b = 0; b < 3; ++b) {
                            T v1 = zero<T>(), v2 = zero<T>(), v3 = zero<T>();
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                v1 = mad(PM(s2, a, c), PM(s3, c, b), v1);   // d/d(M1)_ba -> (M2 M3)_ab
                                v2 = mad(PM(s3, a, c), PM(s1, c, b), v2);   // d/d(M2)_ba -> (M3 M1)_ab
                                v3 = mad(PM(s1, a, c), PM(s2, c, b), v3);   // d/d(M3)_ba -> (M1 M2)_ab
                            }
                            AM(s1, b, a) = mad(g, v1, AM(s1, b, a));
                            AM(s2, b, a) = mad(g, v2, AM(s2, b, a));
                            AM(s3, b, a) = mad(g, v3, AM(s3, b, a));
                        }
                }
    } else if (FAM == 6) {
#pragma unroll
        for (int s1 = 0; s1 < NR; ++s1)
#pragma unroll
            for (int s2 = 0; s2 < NR; ++s2)
                if ((MASK >> s2) & 1)
#pragma unroll
                for (int s3 = s1; s3 < NR; ++s3) {
                    const float g = gb[FAM_OFF6 + f6_index(s1, s2, s3)];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        T w13 = zero<T>(), w31 = zero<T>();
#pragma unroll
                        for (int b = 0; b < 3; ++b) {
                            w13 = mad(PM(s2, a, b), PV(s3, b), w13);
                            w31 = mad(PM(s2, a, b), PV(s1, b), w31);
                            AM(s2, a, b) = mad(g * PV(s1, a), PV(s3, b), AM(s2, a, b));
                        }
                        AV(s1, a) = mad(g, w13, AV(s1, a));
                        AV(s3, a) = mad(g, w31, AV(s3, a));
                    }
                }
    } else if (FAM == 7) {
#pragma unroll
        for (int s1 = 0; s1 < NR; ++s1) {
            if (!((MASK >> s1) & 1)) continue;
#pragma unroll
            for (int s2 = s1; s2 < NR; ++s2) {
                T Mw[3][3], Q[3][3];
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        T v = zero<T>(), w = zero<T>();
#pragma unroll
                        for (int s3 = 0; s3 < NR; ++s3) w = mad(gb[FAM_OFF7 + f7_index(s1, s2, s3)], PM(s3, c, d), w);
#pragma unroll
                        for (int a = 0; a < 3; ++a)
#pragma unroll
                            for (int b = 0; b < 3; ++b) v = mad(PT(s1, a, b, c), PT(s2, a, b, d), v);
                        Mw[c][d] = w;
                        Q[c][d] = v;
                    }
#pragma unroll
                for (int s3 = 0; s3 < NR; ++s3) {
                    const float g = gb[FAM_OFF7 + f7_index(s1, s2, s3)];
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int d = 0; d < 3; ++d) AM(s3, c, d) = mad(g, Q[c][d], AM(s3, c, d));
                }
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b)
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            T t1 = zero<T>(), t2 = zero<T>();
#pragma unroll
                            for (int d = 0; d < 3; ++d) {
                                t1 = mad(PT(s2, a, b, d), Mw[c][d], t1);   // d/d(T1)_abc
                                t2 = mad(PT(s1, a, b, d), Mw[d][c], t2);   // d/d(T2)_abc
                            }
                            AT(s1, a, b, c) += t1;
                            AT(s2, a, b, c) += t2;
                        }
            }
        }
    } else {
#pragma unroll
        for (int s2 = 0; s2 < NR; ++s2) {
            if (!((MASK >> s2) & 1)) continue;
#pragma unroll
            for (int s3 = 0; s3 < NR; ++s3) {
                T U[3], Vw[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    T v = zero<T>(), w = zero<T>();
#pragma unroll
                    for (int b = 0; b < 3; ++b)
#pragma unroll
                        for (int c = 0; c < 3; ++c) v = mad(PT(s2, a, b, c), PM(s3, b, c), v);
#pragma unroll
                    for (int s1 = 0; s1 < NR; ++s1) w = mad(gb[FAM_OFF8 + f8_index(s1, s2, s3)], PV(s1, a), w);
                    U[a] = v;
                    Vw[a] = w;
                }
#pragma unroll
                for (int s1 = 0; s1 < NR; ++s1) {
                    const float g = gb[FAM_OFF8 + f8_index(s1, s2, s3)];
#pragma unroll
                    for (int a = 0; a < 3; ++a) AV(s1, a) = mad(g, U[a], AV(s1, a));
                }
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b)
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            AT(s2, a, b, c) = mad(Vw[a], PM(s3, b, c), AT(s2, a, b, c));
                            AM(s3, b, c) = mad(Vw[a], PT(s2, a, b, c), AM(s3, b, c));
                        }
            }
        }
    }
}

// The eight backward groups of the dual kernel (one warp each), as units.
template <int PART, typename T>
__device__ __forceinline__ void bwd_group(const T (&P)[NPSI], const float *gb, T (&A)[NPSI]) {
    if (PART == 0) bwd_unit<0, 0x1F>(P, gb, A);
    else if (PART == 1) bwd_unit<5, 0x1F>(P, gb, A);
    else if (PART == 2) bwd_unit<6, 0x1F>(P, gb, A);
    else if (PART == 3) bwd_unit<7, 0x01>(P, gb, A);
    else if (PART == 4) bwd_unit<7, 0x12>(P, gb, A);
    else if (PART == 5) bwd_unit<7, 0x0C>(P, gb, A);
    else if (PART == 6) bwd_unit<8, 0x03>(P, gb, A);
    else bwd_unit<8, 0x1C>(P, gb, A);
}

// Eight backward warps of balanced work (estimated FMAs per atom in brackets):
//   #1-#4 + #8 s2=0 [1.7k]; #5 s1 in {0,4} [1.7k]; #5 s1 in {1,2,3} [2.1k]; #6 s2 in {0..3} [2.0k];
//   #7 s1 in {0,4} [2.0k]; #7 s1=1 + #6 s2=4 [1.8k]; #7 s1 in {2,3} + #8 s2=1 [2.2k]; #8 s2 in {2,3,4} [1.7k]
// (eight groups by family alone put 3.8k on the #5 warp).  Nine warps do not fit: at this
// register count one SM sub-partition cannot hold three warps.
constexpr int CT_BWD_WARPS = 8;
template <typename T>
__device__ __forceinline__ void bwd_warp(int warp, const T (&P)[NPSI], const float *gb, T (&A)[NPSI]) {
    switch (warp) {
    case 0: bwd_unit<0, 0x1F>(P, gb, A); bwd_unit<8, 0x01>(P, gb, A); break;
    case 1: bwd_unit<5, 0x11>(P, gb, A); break;
    case 2: bwd_unit<5, 0x0E>(P, gb, A); break;
    case 3: bwd_unit<6, 0x0F>(P, gb, A); break;
    case 4: bwd_unit<7, 0x11>(P, gb, A); break;
    case 5: bwd_unit<7, 0x02>(P, gb, A); bwd_unit<6, 0x10>(P, gb, A); break;
    case 6: bwd_unit<7, 0x0C>(P, gb, A); bwd_unit<8, 0x02>(P, gb, A); break;
    default: bwd_unit<8, 0x1C>(P, gb, A); break;
    }
}

// Stage the 360 leading columns of 32 rows of a [.][384] FP32 matrix into shared memory
// (row stride GT_STRIDE, rows past N zero).  Every thread issues all of its 16-byte loads
// before the first store, so the block waits for one memory latency instead of one per row.
template <int NT>
__device__ __forceinline__ void stage_rows(const float *__restrict__ src, int m0, int N, float *tile) {
    constexpr int V4 = NF / 4, TOT = CT_ATOMS * V4, PER = (TOT + NT - 1) / NT;
    float4 v[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int idx = threadIdx.x + u * NT;
        const int r = idx / V4, q = idx - r * V4;
        v[u] = (idx < TOT && m0 + r < N) ? __ldg(reinterpret_cast<const float4 *>(src + (size_t)(m0 + r) * NFP) + q)
                                         : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int idx = threadIdx.x + u * NT;
        if (idx < TOT) {
            const int r = idx / V4, q = idx - r * V4;
            float *d = tile + r * GT_STRIDE + 4 * q;
            d[0] = v[u].x; d[1] = v[u].y; d[2] = v[u].z; d[3] = v[u].w;
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(CT_BWD_WARPS * 32, 2) k_contract_bwd(const float *__restrict__ psi,
                                                                const float *__restrict__ dG, int N,
                                                                float *__restrict__ dpsi) {
    extern __shared__ float sm[];
    float *gtile = sm;
    float *acc = sm + CT_ATOMS * GT_STRIDE;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * CT_ATOMS;
    stage_rows<CT_BWD_WARPS * 32>(dG, m0, N, gtile);
    float P[NPSI], A[NPSI];
    load_psi(psi, m0 + lane, N, P);
#pragma unroll
    for (int q = 0; q < NPSI; ++q) A[q] = 0.0f;
    const float *gb = gtile + lane * GT_STRIDE;
    bwd_warp(warp, P, gb, A);
    float *arow = acc + lane * AC_STRIDE;
    for (int w = 0; w < CT_BWD_WARPS; ++w) {
        if (warp == w) {
#pragma unroll
            for (int q = 0; q < NPSI; ++q) arow[q] = (w == 0 ? 0.0f : arow[q]) + A[q];
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < CT_ATOMS * NPSI; idx += blockDim.x) {
        const int r = idx / NPSI, q = idx - r * NPSI, m = m0 + r;
        if (m < N) dpsi[(size_t)m * NPSI + q] = acc[r * AC_STRIDE + q];
    }
}

// ------------------------------------------------------------------ parameter-gradient variants
// Dual forward: features G and their tangents Gd = dG/dPsi . Psid, written as the stacked
// GEMM operand GG [2 Mp][384] (rows m: G, rows Mp + m: Gd; FP32).
__global__ void __launch_bounds__(CT_THREADS, 1) k_contract_fwd_dual(const float *__restrict__ psi,
                                                                     const float *__restrict__ psid, int N, int Mp,
                                                                     float *__restrict__ GG) {
    extern __shared__ float tiles[];
    float *tv = tiles, *td = tiles + CT_ATOMS * GT_STRIDE;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * CT_ATOMS;
    Dual P[NPSI];
    {
        float a[NPSI], b[NPSI];
        load_psi(psi, m0 + lane, N, a);
        load_psi(psid, m0 + lane, N, b);
#pragma unroll
        for (int q = 0; q < NPSI; ++q) P[q] = {a[q], b[q]};
    }
    const FeatOut gt{tv + lane * GT_STRIDE, td + lane * GT_STRIDE};
    switch (warp) {
    case 0: fwd_group<0>(P, gt); break;
    case 1: fwd_group<1>(P, gt); break;
    case 2: fwd_group<2>(P, gt); break;
    case 3: fwd_group<3>(P, gt); break;
    case 4: fwd_group<4>(P, gt); break;
    case 5: fwd_group<5>(P, gt); break;
    case 6: fwd_group<6>(P, gt); break;
    default: fwd_group<7>(P, gt); break;
    }
    __syncthreads();
    constexpr int NC4 = NFP / 4;
    for (int idx = threadIdx.x; idx < CT_ATOMS * NC4; idx += CT_THREADS) {
        const int r = idx / NC4, c = idx - r * NC4, m = m0 + r;
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

// Dual backward.  With Gb = dJ/dG and Gdb = dJ/dGd (stacked in Gbs [2 Mp][384]):
//   psib  = J^T Gb + (dJ^T/dPsi . Psid) Gdb   (adjoint of the moments)
//   psidb = J^T Gdb                            (adjoint of the tangent moments)
// where J = dG/dPsi.  The second term is the tangent part of J^T Gdb evaluated on duals.
__global__ void __launch_bounds__(CT_THREADS, 1) k_contract_bwd_dual(const float *__restrict__ psi,
                                                                     const float *__restrict__ psid,
                                                                     const float *__restrict__ Gbs, int N, int Mp,
                                                                     float *__restrict__ psib,
                                                                     float *__restrict__ psidb) {
    extern __shared__ float sm[];
    float *gtile = sm;                                // Gb
    float *gdtile = sm + CT_ATOMS * GT_STRIDE;         // Gdb
    float *acc1 = gdtile + CT_ATOMS * GT_STRIDE;       // psib
    float *acc2 = acc1 + CT_ATOMS * AC_STRIDE;         // psidb
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * CT_ATOMS;
    stage_rows<CT_THREADS>(Gbs, m0, N, gtile);
    stage_rows<CT_THREADS>(Gbs + (size_t)Mp * NFP, m0, N, gdtile);
    float *arow1 = acc1 + lane * AC_STRIDE, *arow2 = acc2 + lane * AC_STRIDE;
    {   // J^T Gb
        float P[NPSI], A[NPSI];
        load_psi(psi, m0 + lane, N, P);
#pragma unroll
        for (int q = 0; q < NPSI; ++q) A[q] = 0.0f;
        const float *gb = gtile + lane * GT_STRIDE;
        switch (warp) {
        case 0: bwd_group<0>(P, gb, A); break;
        case 1: bwd_group<1>(P, gb, A); break;
        case 2: bwd_group<2>(P, gb, A); break;
        case 3: bwd_group<3>(P, gb, A); break;
        case 4: bwd_group<4>(P, gb, A); break;
        case 5: bwd_group<5>(P, gb, A); break;
        case 6: bwd_group<6>(P, gb, A); break;
        default: bwd_group<7>(P, gb, A); break;
        }
        for (int w = 0; w < CT_THREADS / 32; ++w) {
            if (warp == w) {
#pragma unroll
                for (int q = 0; q < NPSI; ++q) arow1[q] = (w == 0 ? 0.0f : arow1[q]) + A[q];
            }
            __syncthreads();
        }
    }
    {   // J^T Gdb on duals: value -> psidb, tangent -> second-order part of psib
        Dual P[NPSI], A[NPSI];
        {
            float a[NPSI], b[NPSI];
            load_psi(psi, m0 + lane, N, a);
            load_psi(psid, m0 + lane, N, b);
#pragma unroll
            for (int q = 0; q < NPSI; ++q) {
                P[q] = {a[q], b[q]};
                A[q] = {0.0f, 0.0f};
            }
        }
        const float *gb = gdtile + lane * GT_STRIDE;
        switch (warp) {
        case 0: bwd_group<0>(P, gb, A); break;
        case 1: bwd_group<1>(P, gb, A); break;
        case 2: bwd_group<2>(P, gb, A); break;
        case 3: bwd_group<3>(P, gb, A); break;
        case 4: bwd_group<4>(P, gb, A); break;
        case 5: bwd_group<5>(P, gb, A); break;
        case 6: bwd_group<6>(P, gb, A); break;
        default: bwd_group<7>(P, gb, A); break;
        }
        for (int w = 0; w < CT_THREADS / 32; ++w) {
            if (warp == w) {
#pragma unroll
                for (int q = 0; q < NPSI; ++q) {
                    arow1[q] += A[q].d;
                    arow2[q] = (w == 0 ? 0.0f : arow2[q]) + A[q].v;
                }
            }
            __syncthreads();
        }
    }
    for (int idx = threadIdx.x; idx < CT_ATOMS * NPSI; idx += CT_THREADS) {
        const int r = idx / NPSI, q = idx - r * NPSI, m = m0 + r;
        if (m < N) {
            psib[(size_t)m * NPSI + q] = acc1[r * AC_STRIDE + q];
            psidb[(size_t)m * NPSI + q] = acc2[r * AC_STRIDE + q];
        }
    }
}

// ------------------------------------------------------------------ launchers
void launch_contract_fwd_dual(const float *psi, const float *psid, int N, int Mp, float *GG, cudaStream_t st) {
    const int blocks = (Mp + CT_ATOMS - 1) / CT_ATOMS;
    const size_t smem = sizeof(float) * 2 * CT_ATOMS * GT_STRIDE;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_contract_fwd_dual, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    if (blocks > 0) {
        k_contract_fwd_dual<<<blocks, CT_THREADS, smem, st>>>(psi, psid, N, Mp, GG);
        note_launches(1);
    }
}

void launch_contract_bwd_dual(const float *psi, const float *psid, const float *Gbs, int N, int Mp, float *psib,
                              float *psidb, cudaStream_t st) {
    const int blocks = (N + CT_ATOMS - 1) / CT_ATOMS;
    const size_t smem = sizeof(float) * (2 * CT_ATOMS * GT_STRIDE + 2 * CT_ATOMS * AC_STRIDE);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_contract_bwd_dual, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    if (blocks > 0) {
        k_contract_bwd_dual<<<blocks, CT_THREADS, smem, st>>>(psi, psid, Gbs, N, Mp, psib, psidb);
        note_launches(1);
    }
}
void launch_contract_fwd_f32(const float *psi, int N, int Mp, float *G, float *features_out, cudaStream_t st) {
    const int blocks = (Mp + CT_ATOMS - 1) / CT_ATOMS;
    const size_t smem = sizeof(float) * CT_ATOMS * GT_STRIDE;
    if (blocks > 0) {
        k_contract_fwd<float><<<blocks, CT_THREADS, smem, st>>>(psi, N, Mp, G, features_out, 0);
        note_launches(1);
    }
}

void launch_contract_fwd_bf16(const float *psi, int N, int Mp, __nv_bfloat16 *G, float *features_out, bool lo_out,
                              cudaStream_t st) {
    const int blocks = (Mp + CT_ATOMS - 1) / CT_ATOMS;
    const size_t smem = sizeof(float) * CT_ATOMS * GT_STRIDE;
    if (blocks > 0) {
        k_contract_fwd<__nv_bfloat16><<<blocks, CT_THREADS, smem, st>>>(psi, N, Mp, G, features_out, lo_out ? 1 : 0);
        note_launches(1);
    }
}

void launch_contract_bwd(const float *psi, const float *dG, int N, float *dpsi, cudaStream_t st) {
    const int blocks = (N + CT_ATOMS - 1) / CT_ATOMS;
    const size_t smem = sizeof(float) * (CT_ATOMS * GT_STRIDE + CT_ATOMS * AC_STRIDE);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_contract_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    if (blocks > 0) {
        k_contract_bwd<<<blocks, CT_BWD_WARPS * 32, smem, st>>>(psi, dG, N, dpsi);
        note_launches(1);
    }
}

}  // namespace gm
