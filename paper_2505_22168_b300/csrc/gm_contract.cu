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
// group w for all 32 atoms, so every warp runs one code path.  Groups: 0 = #1-#4,
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
template <int PART>
__device__ __forceinline__ void fwd_group(const float (&P)[NPSI], float *gt) {
    if (PART == 0) {
#pragma unroll
        for (int s = 0; s < NR; ++s) gt[FAM_OFF1 + s] = P[s * NC];
#pragma unroll
        for (int s1 = 0; s1 < NR; ++s1)
#pragma unroll
            for (int s2 = s1; s2 < NR; ++s2) {
                float f2 = 0.0f, f3 = 0.0f, f4 = 0.0f;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    f2 = fmaf(PV(s1, a), PV(s2, a), f2);
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        f3 = fmaf(PM(s1, a, b), PM(s2, a, b), f3);
#pragma unroll
                        for (int c = 0; c < 3; ++c) f4 = fmaf(PT(s1, a, b, c), PT(s2, a, b, c), f4);
                    }
                }
                const int q = pair_le_index(s1, s2);
                gt[FAM_OFF2 + q] = f2;
                gt[FAM_OFF3 + q] = f3;
                gt[FAM_OFF4 + q] = f4;
            }
    } else if (PART == 1) {
#pragma unroll
        for (int s1 = 0; s1 < NR; ++s1)
#pragma unroll
            for (int s2 = s1; s2 < NR; ++s2) {
                float Nm[3][3];
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        float v = 0.0f;
#pragma unroll
                        for (int b = 0; b < 3; ++b) v = fmaf(PM(s1, a, b), PM(s2, b, c), v);
                        Nm[a][c] = v;
                    }
#pragma unroll
                for (int s3 = s2; s3 < NR; ++s3) {
                    float f = 0.0f;
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int c = 0; c < 3; ++c) f = fmaf(Nm[a][c], PM(s3, c, a), f);
                    gt[FAM_OFF5 + f5_index(s1, s2, s3)] = f;
                }
            }
    } else if (PART == 2) {
#pragma unroll
        for (int s2 = 0; s2 < NR; ++s2)
#pragma unroll
            for (int s3 = 0; s3 < NR; ++s3) {
                float w[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    float v = 0.0f;
#pragma unroll
                    for (int b = 0; b < 3; ++b) v = fmaf(PM(s2, a, b), PV(s3, b), v);
                    w[a] = v;
                }
#pragma unroll
                for (int s1 = 0; s1 <= s3; ++s1) {
                    float f = 0.0f;
#pragma unroll
                    for (int a = 0; a < 3; ++a) f = fmaf(PV(s1, a), w[a], f);
                    gt[FAM_OFF6 + f6_index(s1, s2, s3)] = f;
                }
            }
    } else if (PART >= 3 && PART <= 5) {
#pragma unroll
        for (int s1 = 0; s1 < NR; ++s1) {
            if (!f7_group_has(PART, s1)) continue;
#pragma unroll
            for (int s2 = s1; s2 < NR; ++s2) {
                float Q[3][3];
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        float v = 0.0f;
#pragma unroll
                        for (int a = 0; a < 3; ++a)
#pragma unroll
                            for (int b = 0; b < 3; ++b) v = fmaf(PT(s1, a, b, c), PT(s2, a, b, d), v);
                        Q[c][d] = v;
                    }
#pragma unroll
                for (int s3 = 0; s3 < NR; ++s3) {
                    float f = 0.0f;
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int d = 0; d < 3; ++d) f = fmaf(Q[c][d], PM(s3, c, d), f);
                    gt[FAM_OFF7 + f7_index(s1, s2, s3)] = f;
                }
            }
        }
    } else {
#pragma unroll
        for (int s2 = 0; s2 < NR; ++s2) {
            if (!f8_group_has(PART, s2)) continue;
#pragma unroll
            for (int s3 = 0; s3 < NR; ++s3) {
                float U[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    float v = 0.0f;
#pragma unroll
                    for (int b = 0; b < 3; ++b)
#pragma unroll
                        for (int c = 0; c < 3; ++c) v = fmaf(PT(s2, a, b, c), PM(s3, b, c), v);
                    U[a] = v;
                }
#pragma unroll
                for (int s1 = 0; s1 < NR; ++s1) {
                    float f = 0.0f;
#pragma unroll
                    for (int a = 0; a < 3; ++a) f = fmaf(PV(s1, a), U[a], f);
                    gt[FAM_OFF8 + f8_index(s1, s2, s3)] = f;
                }
            }
        }
    }
}

template <typename OutT>
__device__ __forceinline__ OutT to_out(float v);
template <>
__device__ __forceinline__ float to_out<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_out<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

template <typename OutT>
__global__ void __launch_bounds__(CT_THREADS, 1) k_contract_fwd(const float *__restrict__ psi, int N, int Mp,
                                                                OutT *__restrict__ G, float *__restrict__ G32) {
    extern __shared__ float tile[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * CT_ATOMS;
    float P[NPSI];
    load_psi(psi, m0 + lane, N, P);
    float *gt = tile + lane * GT_STRIDE;
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
    for (int idx = threadIdx.x; idx < CT_ATOMS * NFP; idx += CT_THREADS) {
        const int r = idx / NFP, f = idx - r * NFP, m = m0 + r;
        if (m >= Mp) continue;
        const float v = f < NF ? tile[r * GT_STRIDE + f] : 0.0f;
        if (sizeof(OutT) == 2) {
            // BF16 operand as a hi/lo pair: row [hi(384) | lo(384)]
            const __nv_bfloat16 hi = __float2bfloat16_rn(v);
            const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
            reinterpret_cast<__nv_bfloat16 *>(G)[(size_t)m * 2 * NFP + f] = hi;
            reinterpret_cast<__nv_bfloat16 *>(G)[(size_t)m * 2 * NFP + NFP + f] = lo;
        } else {
            G[(size_t)m * NFP + f] = to_out<OutT>(v);
        }
        if (G32 != nullptr && f < NF && m < N) G32[(size_t)m * NF + f] = v;
    }
}

// ------------------------------------------------------------------ backward groups
template <int PART>
__device__ __forceinline__ void bwd_group(const float (&P)[NPSI], const float *gb, float (&A)[NPSI]) {
    if (PART == 0) {
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
                    AV(s1, a) = fmaf(g2, PV(s2, a), AV(s1, a));
                    AV(s2, a) = fmaf(g2, PV(s1, a), AV(s2, a));
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        AM(s1, a, b) = fmaf(g3, PM(s2, a, b), AM(s1, a, b));
                        AM(s2, a, b) = fmaf(g3, PM(s1, a, b), AM(s2, a, b));
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            AT(s1, a, b, c) = fmaf(g4, PT(s2, a, b, c), AT(s1, a, b, c));
                            AT(s2, a, b, c) = fmaf(g4, PT(s1, a, b, c), AT(s2, a, b, c));
                        }
                    }
                }
            }
    } else if (PART == 1) {
#pragma unroll
        for (int s1 = 0; s1 < NR; ++s1)
#pragma unroll
            for (int s2 = s1; s2 < NR; ++s2)
#pragma unroll
                for (int s3 = s2; s3 < NR; ++s3) {
                    const float g = gb[FAM_OFF5 + f5_index(s1, s2, s3)];
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int b = 0; b < 3; ++b) {
                            float v1 = 0.0f, v2 = 0.0f, v3 = 0.0f;
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                v1 = fmaf(PM(s2, a, c), PM(s3, c, b), v1);   // d/d(M1)_ba -> (M2 M3)_ab
                                v2 = fmaf(PM(s3, a, c), PM(s1, c, b), v2);   // d/d(M2)_ba -> (M3 M1)_ab
                                v3 = fmaf(PM(s1, a, c), PM(s2, c, b), v3);   // d/d(M3)_ba -> (M1 M2)_ab
                            }
                            AM(s1, b, a) = fmaf(g, v1, AM(s1, b, a));
                            AM(s2, b, a) = fmaf(g, v2, AM(s2, b, a));
                            AM(s3, b, a) = fmaf(g, v3, AM(s3, b, a));
                        }
                }
    } else if (PART == 2) {
#pragma unroll
        for (int s1 = 0; s1 < NR; ++s1)
#pragma unroll
            for (int s2 = 0; s2 < NR; ++s2)
#pragma unroll
                for (int s3 = s1; s3 < NR; ++s3) {
                    const float g = gb[FAM_OFF6 + f6_index(s1, s2, s3)];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        float w13 = 0.0f, w31 = 0.0f;
#pragma unroll
                        for (int b = 0; b < 3; ++b) {
                            w13 = fmaf(PM(s2, a, b), PV(s3, b), w13);
                            w31 = fmaf(PM(s2, a, b), PV(s1, b), w31);
                            AM(s2, a, b) = fmaf(g * PV(s1, a), PV(s3, b), AM(s2, a, b));
                        }
                        AV(s1, a) = fmaf(g, w13, AV(s1, a));
                        AV(s3, a) = fmaf(g, w31, AV(s3, a));
                    }
                }
    } else if (PART >= 3 && PART <= 5) {
#pragma unroll
        for (int s1 = 0; s1 < NR; ++s1) {
            if (!f7_group_has(PART, s1)) continue;
#pragma unroll
            for (int s2 = s1; s2 < NR; ++s2) {
                float Mw[3][3], Q[3][3];
#pragma unroll
                for (int c = 0; c < 3; ++c)
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        float v = 0.0f, w = 0.0f;
#pragma unroll
                        for (int s3 = 0; s3 < NR; ++s3) w = fmaf(gb[FAM_OFF7 + f7_index(s1, s2, s3)], PM(s3, c, d), w);
#pragma unroll
                        for (int a = 0; a < 3; ++a)
#pragma unroll
                            for (int b = 0; b < 3; ++b) v = fmaf(PT(s1, a, b, c), PT(s2, a, b, d), v);
                        Mw[c][d] = w;
                        Q[c][d] = v;
                    }
#pragma unroll
                for (int s3 = 0; s3 < NR; ++s3) {
                    const float g = gb[FAM_OFF7 + f7_index(s1, s2, s3)];
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int d = 0; d < 3; ++d) AM(s3, c, d) = fmaf(g, Q[c][d], AM(s3, c, d));
                }
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b)
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            float t1 = 0.0f, t2 = 0.0f;
#pragma unroll
                            for (int d = 0; d < 3; ++d) {
                                t1 = fmaf(PT(s2, a, b, d), Mw[c][d], t1);   // d/d(T1)_abc
                                t2 = fmaf(PT(s1, a, b, d), Mw[d][c], t2);   // d/d(T2)_abc
                            }
                            AT(s1, a, b, c) += t1;
                            AT(s2, a, b, c) += t2;
                        }
            }
        }
    } else {
#pragma unroll
        for (int s2 = 0; s2 < NR; ++s2) {
            if (!f8_group_has(PART, s2)) continue;
#pragma unroll
            for (int s3 = 0; s3 < NR; ++s3) {
                float U[3], Vw[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    float v = 0.0f, w = 0.0f;
#pragma unroll
                    for (int b = 0; b < 3; ++b)
#pragma unroll
                        for (int c = 0; c < 3; ++c) v = fmaf(PT(s2, a, b, c), PM(s3, b, c), v);
#pragma unroll
                    for (int s1 = 0; s1 < NR; ++s1) w = fmaf(gb[FAM_OFF8 + f8_index(s1, s2, s3)], PV(s1, a), w);
                    U[a] = v;
                    Vw[a] = w;
                }
#pragma unroll
                for (int s1 = 0; s1 < NR; ++s1) {
                    const float g = gb[FAM_OFF8 + f8_index(s1, s2, s3)];
#pragma unroll
                    for (int a = 0; a < 3; ++a) AV(s1, a) = fmaf(g, U[a], AV(s1, a));
                }
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b)
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            AT(s2, a, b, c) = fmaf(Vw[a], PM(s3, b, c), AT(s2, a, b, c));
                            AM(s3, b, c) = fmaf(Vw[a], PT(s2, a, b, c), AM(s3, b, c));
                        }
            }
        }
    }
}

__global__ void __launch_bounds__(CT_THREADS, 1) k_contract_bwd(const float *__restrict__ psi,
                                                                const float *__restrict__ dG, int N,
                                                                float *__restrict__ dpsi) {
    extern __shared__ float sm[];
    float *gtile = sm;
    float *acc = sm + CT_ATOMS * GT_STRIDE;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * CT_ATOMS;
    for (int idx = threadIdx.x; idx < CT_ATOMS * NF; idx += CT_THREADS) {
        const int r = idx / NF, f = idx - r * NF, m = m0 + r;
        gtile[r * GT_STRIDE + f] = m < N ? dG[(size_t)m * NFP + f] : 0.0f;
    }
    __syncthreads();
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
    float *arow = acc + lane * AC_STRIDE;
    for (int w = 0; w < CT_THREADS / 32; ++w) {
        if (warp == w) {
#pragma unroll
            for (int q = 0; q < NPSI; ++q) arow[q] = (w == 0 ? 0.0f : arow[q]) + A[q];
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < CT_ATOMS * NPSI; idx += CT_THREADS) {
        const int r = idx / NPSI, q = idx - r * NPSI, m = m0 + r;
        if (m < N) dpsi[(size_t)m * NPSI + q] = acc[r * AC_STRIDE + q];
    }
}

// ------------------------------------------------------------------ launchers
void launch_contract_fwd_f32(const float *psi, int N, int Mp, float *G, float *features_out, cudaStream_t st) {
    const int blocks = (Mp + CT_ATOMS - 1) / CT_ATOMS;
    const size_t smem = sizeof(float) * CT_ATOMS * GT_STRIDE;
    if (blocks > 0) {
        k_contract_fwd<float><<<blocks, CT_THREADS, smem, st>>>(psi, N, Mp, G, features_out);
        note_launches(1);
    }
}

void launch_contract_fwd_bf16(const float *psi, int N, int Mp, __nv_bfloat16 *G, float *features_out,
                              cudaStream_t st) {
    const int blocks = (Mp + CT_ATOMS - 1) / CT_ATOMS;
    const size_t smem = sizeof(float) * CT_ATOMS * GT_STRIDE;
    if (blocks > 0) {
        k_contract_fwd<__nv_bfloat16><<<blocks, CT_THREADS, smem, st>>>(psi, N, Mp, G, features_out);
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
        k_contract_bwd<<<blocks, CT_THREADS, smem, st>>>(psi, dG, N, dpsi);
        note_launches(1);
    }
}

}  // namespace gm
