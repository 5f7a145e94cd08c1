// gm_pgrad.cu -- network part of the force-matching parameter gradient (FP32).
//
// Objective per atom: j_i = c_i E_i - dE_i/dt, with c_i = dL/dE of its structure and
// d/dt the derivative when positions move along v = dL/dF (sum_i v_i . F_i = -dE/dt).
// Rows m of the stacked [2 Mp][H] arrays hold primal quantities, rows Mp + m their
// tangents.  Activation derivatives phi', phi'' are kept from the forward pass.
//   act1:   a1 = phi(z1 + b1), da1 = phi'(.) dz1                     (forward, layer 1)
//   act2:   a2, da2; NN = w3.a2 + b3, dNN = w3.da2; then the reverse of
//           E = sigma NN + mu, dE = sigma dNN with weights (c, -1):
//           a2b = c sigma w3, da2b = -sigma w3
//           dz2b = phi'(z2) da2b,  z2b = phi''(z2) dz2 da2b + phi'(z2) a2b
//   act1b:  dz1b = phi'(z1) da1b, z1b = phi''(z1) dz1 da1b + phi'(z1) a1b
// Weight gradients: dW = X^T Y over the stacked rows (primal and tangent terms), split
// over K = 2 Mp and summed in fixed order; bias gradients are column sums.
#include "gm_pgrad.h"

namespace gm {

template <int ACT>
__global__ void __launch_bounds__(256) k_pg_act1(int Mp, int H, const float *__restrict__ Z,
                                                 const float *__restrict__ b1, float *__restrict__ A1s,
                                                 float *__restrict__ P1, float *__restrict__ Q1,
                                                 float *__restrict__ Zd1) {
    const size_t n = (size_t)Mp * H;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int h = (int)(q % H);
        const float z = Z[q] + b1[h], zd = Z[n + q];
        float d1, d2;
        const float a = act_fwd2<ACT>(z, d1, d2);
        A1s[q] = a;
        A1s[n + q] = d1 * zd;
        P1[q] = d1;
        Q1[q] = d2;
        Zd1[q] = zd;
    }
}

// one warp per atom row
template <int ACT>
__global__ void __launch_bounds__(256) k_pg_act2(int N, int Mp, int H, int B, const int32_t *__restrict__ atom_ptr,
                                                 const int32_t *__restrict__ species, int S,
                                                 const double *__restrict__ gE, const float *__restrict__ sigma,
                                                 const float *__restrict__ w3, const float *__restrict__ b2,
                                                 const float *__restrict__ b3, const float *__restrict__ Z,
                                                 float *__restrict__ Zb2s, float *__restrict__ Y3,
                                                 float *__restrict__ t_sig, float *__restrict__ t_c,
                                                 float *__restrict__ t_cs) {
    const int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (m >= Mp) return;
    const size_t n = (size_t)Mp * H;
    float c = 0.0f, sg = 0.0f;
    if (m < N) {
        c = (float)gE[structure_of(atom_ptr, B, m)];
        sg = sigma[min(max(species[m], 0), S - 1)];
    }
    float nn = 0.0f, nnd = 0.0f;
    for (int h = lane; h < H; h += 32) {
        const size_t q = (size_t)m * H + h;
        const float z = Z[q] + b2[h], zd = Z[n + q];
        float d1, d2;
        const float a = act_fwd2<ACT>(z, d1, d2);
        const float ad = d1 * zd;
        const float w = w3[h];
        nn = fmaf(w, a, nn);
        nnd = fmaf(w, ad, nnd);
        const float a2b = c * sg * w, da2b = -sg * w;
        Zb2s[q] = d2 * zd * da2b + d1 * a2b;
        Zb2s[n + q] = d1 * da2b;
        Y3[q] = c * sg * a - sg * ad;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        nn += __shfl_xor_sync(0xffffffffu, nn, off);
        nnd += __shfl_xor_sync(0xffffffffu, nnd, off);
    }
    if (lane == 0) {
        t_sig[m] = m < N ? c * (nn + b3[0]) - nnd : 0.0f;
        t_c[m] = m < N ? c : 0.0f;
        t_cs[m] = m < N ? c * sg : 0.0f;
    }
}

__global__ void __launch_bounds__(256) k_pg_act1b(int Mp, int H, const float *__restrict__ Ab,
                                                  const float *__restrict__ P1, const float *__restrict__ Q1,
                                                  const float *__restrict__ Zd1, float *__restrict__ Zb1s) {
    const size_t n = (size_t)Mp * H;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const float ab = Ab[q], adb = Ab[n + q], p = P1[q];
        Zb1s[q] = Q1[q] * Zd1[q] * adb + p * ab;
        Zb1s[n + q] = p * adb;
    }
}

// out[h] = sum_{m < M} A[m][h], one thread per column (fixed order, FP64 accumulation)
__global__ void __launch_bounds__(256) k_colsum(int M, int H, const float *__restrict__ A, float *__restrict__ out) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= H) return;
    double s = 0.0;
    for (int m = 0; m < M; ++m) s += A[(size_t)m * H + h];
    out[h] = (float)s;
}

// C_part[z][i][j] = sum_{k in slice z} A[k][i] B[k][j]; 64 x 64 tiles, 4 x 4 per thread
constexpr int WG_T = 64, WG_K = 16;
__global__ void __launch_bounds__(256) k_wgrad(const float *__restrict__ A, int lda, const float *__restrict__ Bm,
                                               int ldb, int K, int Mo, int No, int kchunk, float *__restrict__ part) {
    __shared__ float As[WG_K][WG_T], Bs[WG_K][WG_T];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int i0 = blockIdx.x * WG_T, j0 = blockIdx.y * WG_T, z = blockIdx.z;
    const int kb = z * kchunk, ke = min(K, kb + kchunk);
    float acc[4][4] = {};
    for (int k0 = kb; k0 < ke; k0 += WG_K) {
        for (int e = tid; e < WG_K * WG_T; e += 256) {
            const int kk = e / WG_T, ii = e % WG_T, k = k0 + kk;
            As[kk][ii] = (k < ke && i0 + ii < Mo) ? A[(size_t)k * lda + i0 + ii] : 0.0f;
            Bs[kk][ii] = (k < ke && j0 + ii < No) ? Bm[(size_t)k * ldb + j0 + ii] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < WG_K; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[kk][ty * 4 + q];
                b[q] = Bs[kk][tx * 4 + q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + ty * 4 + p, j = j0 + tx * 4 + q;
            if (i < Mo && j < No) part[((size_t)z * Mo + i) * No + j] = acc[p][q];
        }
}

__global__ void __launch_bounds__(256) k_wgrad_reduce(int ksplit, int Mo, int No, int Mstore,
                                                      const float *__restrict__ part, float *__restrict__ out) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)Mstore * No) return;
    double s = 0.0;
    for (int z = 0; z < ksplit; ++z) s += part[(size_t)z * Mo * No + e];
    out[e] = (float)s;
}

// per-species sums of the scale/shift gradients and the output bias (one block)
__global__ void __launch_bounds__(256) k_pg_tail(int N, const int32_t *__restrict__ species, int S,
                                                 const float *__restrict__ t_sig, const float *__restrict__ t_c,
                                                 const float *__restrict__ t_cs, float *g_sigma, float *g_mu,
                                                 float *g_b3) {
    __shared__ double sh[256];
    for (int z = -1; z < S; ++z) {
        for (int which = 0; which < (z < 0 ? 1 : 2); ++which) {
            double v = 0.0;
            for (int i = threadIdx.x; i < N; i += blockDim.x) {
                if (z < 0) v += t_cs[i];
                else if (min(max(species[i], 0), S - 1) == z) v += which == 0 ? t_sig[i] : t_c[i];
            }
            sh[threadIdx.x] = v;
            __syncthreads();
            if (threadIdx.x == 0) {
                double s = 0.0;
                for (int q = 0; q < (int)blockDim.x; ++q) s += sh[q];
                if (z < 0) *g_b3 = (float)s;
                else if (which == 0) g_sigma[z] = (float)s;
                else g_mu[z] = (float)s;
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(256) k_pg_beta_reduce(int nblocks, int nbeta, float scale,
                                                        const float *__restrict__ part, float *__restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nbeta) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * nbeta + e];
    out[e] = (float)(s * scale);
}

// ------------------------------------------------------------------ launchers
void pg_act1(int act, int Mp, int H, const float *Z, const float *b1, float *A1s, float *P1, float *Q1, float *Zd1,
             cudaStream_t st) {
    const int blocks = 148 * 8;
    if (act == 0) k_pg_act1<0><<<blocks, 256, 0, st>>>(Mp, H, Z, b1, A1s, P1, Q1, Zd1);
    else k_pg_act1<1><<<blocks, 256, 0, st>>>(Mp, H, Z, b1, A1s, P1, Q1, Zd1);
    note_launches(1);
}

void pg_act2(int act, int N, int Mp, int H, int B, const int32_t *atom_ptr, const int32_t *species, int S,
             const double *gE, const float *sigma, const float *w3, const float *b2, const float *b3, const float *Z,
             float *Zb2s, float *Y3, float *t_sig, float *t_c, float *t_cs, cudaStream_t st) {
    const int blocks = (Mp * 32 + 255) / 256;
    if (act == 0)
        k_pg_act2<0><<<blocks, 256, 0, st>>>(N, Mp, H, B, atom_ptr, species, S, gE, sigma, w3, b2, b3, Z, Zb2s, Y3,
                                             t_sig, t_c, t_cs);
    else
        k_pg_act2<1><<<blocks, 256, 0, st>>>(N, Mp, H, B, atom_ptr, species, S, gE, sigma, w3, b2, b3, Z, Zb2s, Y3,
                                             t_sig, t_c, t_cs);
    note_launches(1);
}

void pg_act1b(int Mp, int H, const float *Ab, const float *P1, const float *Q1, const float *Zd1, float *Zb1s,
              cudaStream_t st) {
    k_pg_act1b<<<148 * 8, 256, 0, st>>>(Mp, H, Ab, P1, Q1, Zd1, Zb1s);
    note_launches(1);
}

void colsum(int M, int H, const float *A, float *out, cudaStream_t st) {
    k_colsum<<<(H + 255) / 256, 256, 0, st>>>(M, H, A, out);
    note_launches(1);
}

int wgrad_ksplit(int K) {
    int ks = K / 1024;
    return ks < 1 ? 1 : (ks > 64 ? 64 : ks);
}

void wgrad(const float *A, int lda, const float *B, int ldb, int K, int Mo, int No, int Mstore, float *part, float *out,
           cudaStream_t st) {
    const int ks = wgrad_ksplit(K);
    int kchunk = (K + ks - 1) / ks;
    kchunk = (kchunk + WG_K - 1) / WG_K * WG_K;
    dim3 grid((Mo + WG_T - 1) / WG_T, (No + WG_T - 1) / WG_T, ks);
    k_wgrad<<<grid, 256, 0, st>>>(A, lda, B, ldb, K, Mo, No, kchunk, part);
    const size_t n = (size_t)Mstore * No;
    k_wgrad_reduce<<<(int)((n + 255) / 256), 256, 0, st>>>(ks, Mo, No, Mstore, part, out);
    note_launches(2);
}

void pg_tail(int N, const int32_t *species, int S, const float *t_sig, const float *t_c, const float *t_cs,
             float *g_sigma, float *g_mu, float *g_b3, cudaStream_t st) {
    k_pg_tail<<<1, 256, 0, st>>>(N, species, S, t_sig, t_c, t_cs, g_sigma, g_mu, g_b3);
    note_launches(1);
}

void pg_beta_reduce(int nblocks, int nbeta, float scale, const float *part, float *out, cudaStream_t st) {
    k_pg_beta_reduce<<<(nbeta + 255) / 256, 256, 0, st>>>(nblocks, nbeta, scale, part, out);
    note_launches(1);
}

}  // namespace gm
