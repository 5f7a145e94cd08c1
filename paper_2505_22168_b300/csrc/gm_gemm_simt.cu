// gm_gemm_simt.cu -- FP32 register-tiled GEMM (FFMA) with the network epilogues; the
// plain-FP32 comparison path (TF32 would not meet a 1e-5 relative tolerance).
//
// Tile 128 x 64 x 16, 256 threads, 8 x 4 outputs per thread, shared-memory double
// buffer fed through registers (one barrier per k-step).
#include "gm_gemm.h"

namespace gm {

constexpr int SB_M = 128, SB_N = 64, SB_K = 16;

template <int EPI, int ACT>
__global__ void __launch_bounds__(256) k_gemm_f32(const float *__restrict__ A, const float *__restrict__ B, int M,
                                                  int N, int K, EpiArgs e) {
    griddep_wait();
    __shared__ __align__(16) float As[2][SB_K][SB_M + 4];
    __shared__ __align__(16) float Bs[2][SB_K][SB_N + 4];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    // the N tiles of one row block are consecutive blocks, so the A rows come from DRAM once
    const int m0 = blockIdx.y * SB_M, n0 = blockIdx.x * SB_N;
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;

    const int ar0 = tid >> 2, akq = (tid & 3) * 4;  // A rows ar0 and ar0 + 64
    const int br = tid >> 2, bkq = (tid & 3) * 4;
    const float *Ap0 = A + (size_t)(m0 + ar0) * K + akq;
    const float *Ap1 = A + (size_t)(m0 + ar0 + 64) * K + akq;
    const float *Bp = B + (size_t)(n0 + br) * K + bkq;
    float4 ra0 = *reinterpret_cast<const float4 *>(Ap0);
    float4 ra1 = *reinterpret_cast<const float4 *>(Ap1);
    float4 rb = *reinterpret_cast<const float4 *>(Bp);
    auto stash = [&](int buf) {
        As[buf][akq + 0][ar0] = ra0.x; As[buf][akq + 1][ar0] = ra0.y;
        As[buf][akq + 2][ar0] = ra0.z; As[buf][akq + 3][ar0] = ra0.w;
        As[buf][akq + 0][ar0 + 64] = ra1.x; As[buf][akq + 1][ar0 + 64] = ra1.y;
        As[buf][akq + 2][ar0 + 64] = ra1.z; As[buf][akq + 3][ar0 + 64] = ra1.w;
        Bs[buf][bkq + 0][br] = rb.x; Bs[buf][bkq + 1][br] = rb.y;
        Bs[buf][bkq + 2][br] = rb.z; Bs[buf][bkq + 3][br] = rb.w;
    };
    stash(0);
    __syncthreads();
    int cur = 0;
    for (int k0 = 0; k0 < K; k0 += SB_K) {
        const bool more = k0 + SB_K < K;
        if (more) {
            ra0 = *reinterpret_cast<const float4 *>(Ap0 + k0 + SB_K);
            ra1 = *reinterpret_cast<const float4 *>(Ap1 + k0 + SB_K);
            rb = *reinterpret_cast<const float4 *>(Bp + k0 + SB_K);
        }
#pragma unroll
        for (int kk = 0; kk < SB_K; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[cur][kk][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[cur][kk][ty * 8 + 4]);
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[cur][kk][tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (more) stash(cur ^ 1);
        __syncthreads();
        cur ^= 1;
    }

    // ---- epilogue
    const int nb = n0 + tx * 4;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = m0 + ty * 8 + i;
        float *o0 = static_cast<float *>(e.out0) + (size_t)m * N + nb;
        if (EPI == EPI_STORE) {
            *reinterpret_cast<float4 *>(o0) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        } else if (EPI == EPI_B1) {
            const int ma = e.aux_rows ? m % e.aux_rows : m;
            const float4 d = *reinterpret_cast<const float4 *>(static_cast<const float *>(e.aux) + (size_t)ma * N + nb);
            *reinterpret_cast<float4 *>(o0) = make_float4(acc[i][0] * d.x, acc[i][1] * d.y, acc[i][2] * d.z, acc[i][3] * d.w);
        } else if (EPI == EPI_L1) {
            float a[4], d[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) a[j] = act_fwd<ACT>(acc[i][j] + e.bias[nb + j], d[j]);
            *reinterpret_cast<float4 *>(o0) = make_float4(a[0], a[1], a[2], a[3]);
            float *o1 = static_cast<float *>(e.out1) + (size_t)m * N + nb;
            *reinterpret_cast<float4 *>(o1) = make_float4(d[0], d[1], d[2], d[3]);
        } else if (EPI == EPI_L2H) {
            const float sg = m < e.n_atoms ? e.sigma[min(max(e.species[m], 0), e.n_species - 1)] : 0.0f;
            float y[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float d;
                act_fwd<ACT>(acc[i][j] + e.bias[nb + j], d);
                y[j] = sg * d;
            }
            for (int k = 0; k < e.n_heads; ++k) {
                const float4 w = *reinterpret_cast<const float4 *>(e.w3 + (size_t)k * N + nb);
                *reinterpret_cast<float4 *>(o0 + k * e.head_stride) = make_float4(y[0] * w.x, y[1] * w.y, y[2] * w.z, y[3] * w.w);
            }
        } else {  // EPI_L2, EPI_L2E
            const float sg = m < e.n_atoms ? e.sigma[min(max(e.species[m], 0), e.n_species - 1)] : 0.0f;
            float part = 0.0f, dz[4], av[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float d;
                const float a = act_fwd<ACT>(acc[i][j] + e.bias[nb + j], d);
                const float w = e.w3[nb + j];
                part = fmaf(a, w, part);
                dz[j] = sg * w * d;
                av[j] = a;
            }
            *reinterpret_cast<float4 *>(o0) = make_float4(dz[0], dz[1], dz[2], dz[3]);
#pragma unroll
            for (int off = 4; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
            if ((tx & 7) == 0) e.nn_part[(size_t)m * (N / 32) + (n0 + tx * 4) / 32] = part;
            if (EPI == EPI_L2E) {
                for (int k = 0; k < e.n_ens; ++k) {
                    const float *wk = e.w3e + (size_t)k * N + nb;
                    float p = 0.0f;
#pragma unroll
                    for (int j = 0; j < 4; ++j) p = fmaf(av[j], wk[j], p);
#pragma unroll
                    for (int off = 4; off > 0; off >>= 1) p += __shfl_xor_sync(0xffffffffu, p, off);
                    if ((tx & 7) == 0) e.nn_ens[((size_t)k * (N / 32) + (n0 + tx * 4) / 32) * e.nn_ens_ld + m] = p;
                }
            }
        }
    }
}

template <int EPI>
static void launch_act(int act, dim3 g, const float *A, const float *B, int M, int N, int K, const EpiArgs &e,
                       cudaStream_t st) {
    if (act == 0) launch_pdl(k_gemm_f32<EPI, 0>, g, dim3(256), 0, st, A, B, M, N, K, e);
    else launch_pdl(k_gemm_f32<EPI, 1>, g, dim3(256), 0, st, A, B, M, N, K, e);
}

void gemm_f32(int epi, int act, const float *A, const float *B, int M, int N, int K, const EpiArgs &e,
              cudaStream_t st) {
    if (M <= 0) return;
    dim3 g(N / SB_N, M / SB_M);
    note_launches(1);
    switch (epi) {
    case EPI_L1: launch_act<EPI_L1>(act, g, A, B, M, N, K, e, st); break;
    case EPI_L2: launch_act<EPI_L2>(act, g, A, B, M, N, K, e, st); break;
    case EPI_L2E: launch_act<EPI_L2E>(act, g, A, B, M, N, K, e, st); break;
    case EPI_L2H: launch_act<EPI_L2H>(act, g, A, B, M, N, K, e, st); break;
    case EPI_B1: launch_pdl(k_gemm_f32<EPI_B1, 0>, g, dim3(256), 0, st, A, B, M, N, K, e); break;
    default: launch_pdl(k_gemm_f32<EPI_STORE, 0>, g, dim3(256), 0, st, A, B, M, N, K, e); break;
    }
}

}  // namespace gm
