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

// Fixed-order compensated FP32 summation (Kahan): a few ulps of error whatever the number of
// terms, at FP32 speed (B300 issues FP64 adds at a small fraction of the FP32 rate).
struct KahanSum {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c, t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// The mixed path's next GEMM reads its A operand as hi/lo BF16 rows [hi(H) | lo(H)] of the
// stacked [2 Mp] rows: the kernels that produce that operand write the copy as well (hl, or
// null in the FP32 path), instead of a separate conversion pass.
__device__ __forceinline__ void put_split(__nv_bfloat16 *hl, size_t row, int h, int H, float x) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
    hl[row * 2 * H + h] = hi;
    hl[row * 2 * H + H + h] = __float2bfloat16_rn(x - __bfloat162float(hi));
}

template <int ACT>
__global__ void __launch_bounds__(256) k_pg_act1(int Mp, int H, const float *__restrict__ Z,
                                                 const float *__restrict__ b1, float *__restrict__ A1s,
                                                 float *__restrict__ P1, float *__restrict__ Q1,
                                                 float *__restrict__ Zd1, __nv_bfloat16 *__restrict__ hl) {
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
        if (hl) {
            const size_t m = q / H;
            put_split(hl, m, h, H, a);
            put_split(hl, Mp + m, h, H, d1 * zd);
        }
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
                                                 float *__restrict__ t_cs, __nv_bfloat16 *__restrict__ hl) {
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
        const float zb = d2 * zd * da2b + d1 * a2b, zbd = d1 * da2b;
        Zb2s[q] = zb;
        Zb2s[n + q] = zbd;
        Y3[q] = c * sg * a - sg * ad;
        if (hl) {
            put_split(hl, m, h, H, zb);
            put_split(hl, Mp + m, h, H, zbd);
        }
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
                                                  const float *__restrict__ Zd1, float *__restrict__ Zb1s,
                                                  __nv_bfloat16 *__restrict__ hl) {
    const size_t n = (size_t)Mp * H;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const float ab = Ab[q], adb = Ab[n + q], p = P1[q];
        const float zb = Q1[q] * Zd1[q] * adb + p * ab, zbd = p * adb;
        Zb1s[q] = zb;
        Zb1s[n + q] = zbd;
        if (hl) {
            const size_t m = q / H;
            const int h = (int)(q - m * H);
            put_split(hl, m, h, H, zb);
            put_split(hl, Mp + m, h, H, zbd);
        }
    }
}

// Column sums out_a[h] = sum_{m < M} A_a[m][h] of up to three arrays A_a [M][H] in one launch
// pair: block (column group of 32, chunk of CS_ROWS rows, array a) writes
// part[a][chunk][col]; k_colsum_final adds the chunks in a fixed order (compensated).
constexpr int CS_ROWS = 256;
struct ColSums {
    const float *A[3];
    float *out[3];
};
__global__ void __launch_bounds__(256) k_colsum_part(int M, int H, ColSums cs, float *__restrict__ part) {
    __shared__ float sm[8][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int col = blockIdx.x * 32 + lane;
    const int r0 = blockIdx.y * CS_ROWS, r1 = min(M, r0 + CS_ROWS);
    const float *__restrict__ A = cs.A[blockIdx.z];
    float s = 0.0f;
    if (col < H)
        for (int m = r0 + warp; m < r1; m += 8) s += A[(size_t)m * H + col];
    sm[warp][lane] = s;
    __syncthreads();
    if (warp == 0 && col < H) {
        float t = 0.0f;
#pragma unroll
        for (int w = 0; w < 8; ++w) t += sm[w][lane];
        part[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * H + col] = t;
    }
}

// 32 columns per block: thread group g (threadIdx.y) adds chunks g, g + 8, ... in order, then
// the eight group sums are added in group order (both compensated): a fixed order.
__global__ void __launch_bounds__(256) k_colsum_final(int chunks, int H, ColSums cs, const float *__restrict__ part) {
    __shared__ float sm[8][32];
    const int h = blockIdx.x * 32 + threadIdx.x;
    KahanSum k;
    if (h < H)
#pragma unroll 4
        for (int r = threadIdx.y; r < chunks; r += 8) k.add(part[((size_t)blockIdx.y * chunks + r) * H + h]);
    sm[threadIdx.y][threadIdx.x] = k.s - k.c;
    __syncthreads();
    if (threadIdx.y == 0 && h < H) {
        KahanSum t;
#pragma unroll
        for (int g = 0; g < 8; ++g) t.add(sm[g][threadIdx.x]);
        cs.out[blockIdx.y][h] = t.s;
    }
}

// C_part[z][i][j] = sum_{k in slice z} A[k][i] B[k][j] (A [K][lda], B [K][ldb], row-major):
// 128 x 128 tiles, 8 x 8 per thread (rows 4 ty + {0..3} and 64 + 4 ty + {0..3}, columns
// likewise), 8 rows of K per step staged in shared memory; the next step's 16-byte global
// loads are in flight while the current step is multiplied.  Mo and No are multiples of 4.
constexpr int WG_T = 128, WG_K = 8;
__global__ void __launch_bounds__(256) k_wgrad(const float *__restrict__ A, int lda, const float *__restrict__ Bm,
                                               int ldb, int K, int Mo, int No, int kchunk, float *__restrict__ part) {
    __shared__ __align__(16) float As[2][WG_K][WG_T], Bs[2][WG_K][WG_T];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int i0 = blockIdx.x * WG_T, j0 = blockIdx.y * WG_T, z = blockIdx.z;
    const int kb = z * kchunk, ke = min(K, kb + kchunk);
    const int lr = tid >> 5, lc = (tid & 31) * 4;                 // this thread's 16-byte load in a step
    const float4 zero4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float4 av = zero4, bv = zero4;
    auto fetch = [&](int k0) {
        const int k = k0 + lr;
        av = (k < ke && i0 + lc < Mo) ? __ldg(reinterpret_cast<const float4 *>(A + (size_t)k * lda + i0 + lc)) : zero4;
        bv = (k < ke && j0 + lc < No) ? __ldg(reinterpret_cast<const float4 *>(Bm + (size_t)k * ldb + j0 + lc)) : zero4;
    };
    float acc[8][8];
#pragma unroll
    for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[p][q] = 0.0f;
    fetch(kb);
    int buf = 0;
    for (int k0 = kb; k0 < ke; k0 += WG_K) {
        *reinterpret_cast<float4 *>(&As[buf][lr][lc]) = av;
        *reinterpret_cast<float4 *>(&Bs[buf][lr][lc]) = bv;
        __syncthreads();
        if (k0 + WG_K < ke) fetch(k0 + WG_K);
#pragma unroll
        for (int kk = 0; kk < WG_K; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][4 * ty]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][64 + 4 * ty]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][4 * tx]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + 4 * tx]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int p = 0; p < 8; ++p)
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
        }
        buf ^= 1;
    }
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        const int i = i0 + (p < 4 ? 4 * ty + p : 64 + 4 * ty + p - 4);
        if (i >= Mo) continue;
        float *row = part + ((size_t)z * Mo + i) * No;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = j0 + h * 64 + 4 * tx;
            if (j < No)
                *reinterpret_cast<float4 *>(row + j) =
                    make_float4(acc[p][4 * h], acc[p][4 * h + 1], acc[p][4 * h + 2], acc[p][4 * h + 3]);
        }
    }
}

// The K slices of 32 consecutive outputs per block: thread group g (threadIdx.y) adds slices
// g, g + 8, ... in slice order, then the eight group sums are added in group order (both
// compensated, KahanSum): a fixed order, so the result is the same on every run.
constexpr int WR_OUT = 32, WR_GRP = 8;
__global__ void __launch_bounds__(WR_OUT * WR_GRP) k_wgrad_reduce(int ksplit, int Mo, int No, int Mstore,
                                                                 const float *__restrict__ part,
                                                                 float *__restrict__ out) {
    __shared__ float sm[WR_GRP][WR_OUT];
    const size_t e = (size_t)blockIdx.x * WR_OUT + threadIdx.x, n = (size_t)Mstore * No;
    KahanSum k;
    if (e < n)
#pragma unroll 4
        for (int z = threadIdx.y; z < ksplit; z += WR_GRP) k.add(__ldg(part + (size_t)z * Mo * No + e));
    sm[threadIdx.y][threadIdx.x] = k.s - k.c;
    __syncthreads();
    if (threadIdx.y == 0 && e < n) {
        KahanSum t;
#pragma unroll
        for (int g = 0; g < WR_GRP; ++g) t.add(sm[g][threadIdx.x]);
        out[e] = t.s;
    }
}

// Per-species sums of the scale/shift gradients and the output-bias sum: block b sums the
// atoms [b * TAIL_ATOMS, ...) into part[b][q], q = 0 (b3), 1 + z (sigma_z), 1 + S + z (mu_z);
// k_pg_tail_final adds the blocks in a fixed order (compensated).
constexpr int TAIL_ATOMS = 256;
__global__ void __launch_bounds__(256) k_pg_tail_part(int N, const int32_t *__restrict__ species, int S,
                                                      const float *__restrict__ t_sig, const float *__restrict__ t_c,
                                                      const float *__restrict__ t_cs, float *__restrict__ part) {
    __shared__ float sm[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int a0 = blockIdx.x * TAIL_ATOMS, a1 = min(N, a0 + TAIL_ATOMS);
    const int nq = 1 + 2 * S;
    for (int q = 0; q < nq; ++q) {
        const int z = q == 0 ? -1 : (q - 1) % S;
        const bool mu = q > S;
        float v = 0.0f;
        for (int i = a0 + threadIdx.x; i < a1; i += blockDim.x) {
            if (z < 0) v += t_cs[i];
            else if (min(max(species[i], 0), S - 1) == z) v += mu ? t_c[i] : t_sig[i];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sm[warp] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.0f;
            for (int w = 0; w < 8; ++w) t += sm[w];
            part[(size_t)blockIdx.x * nq + q] = t;
        }
        __syncthreads();
    }
}

__global__ void k_pg_tail_final(int nblocks, int S, const float *__restrict__ part, float *g_sigma, float *g_mu,
                                float *g_b3) {
    const int q = threadIdx.x, nq = 1 + 2 * S;
    if (q >= nq) return;
    KahanSum k;
#pragma unroll 8
    for (int b = 0; b < nblocks; ++b) k.add(part[(size_t)b * nq + q]);
    if (q == 0) *g_b3 = k.s;
    else if (q <= S) g_sigma[q - 1] = k.s;
    else g_mu[q - 1 - S] = k.s;
}

// One warp per coefficient: lanes take every 32nd block partial (compensated), then a fixed
// shuffle tree adds the lanes' sums.
__global__ void __launch_bounds__(256) k_pg_beta_reduce(int nblocks, int nbeta, float scale,
                                                        const float *__restrict__ part, float *__restrict__ out) {
    const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (e >= nbeta) return;
    KahanSum k;
#pragma unroll 4
    for (int b = lane; b < nblocks; b += 32) k.add(part[(size_t)b * nbeta + e]);
    float s = k.s;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[e] = s * scale;
}

// hi/lo BF16 copy of an FP32 matrix [rows][K]: dst row = [hi(K) | lo(K)], lo = bf16(x - hi)
__global__ void __launch_bounds__(256) k_split_bf16(const float *__restrict__ src, int rows, int K,
                                                    __nv_bfloat16 *__restrict__ dst) {
    const int kw = K / 8;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)rows * kw) return;
    const size_t r = idx / kw;
    const int c = (int)(idx - r * kw) * 8;
    const float4 v0 = *reinterpret_cast<const float4 *>(src + r * K + c);
    const float4 v1 = *reinterpret_cast<const float4 *>(src + r * K + c + 4);
    const float v[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
    __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        hi[q] = __float2bfloat16_rn(v[q]);
        lo[q] = __float2bfloat16_rn(v[q] - __bfloat162float(hi[q]));
    }
    *reinterpret_cast<uint4 *>(dst + r * 2 * K + c) = *reinterpret_cast<const uint4 *>(hi);
    *reinterpret_cast<uint4 *>(dst + r * 2 * K + K + c) = *reinterpret_cast<const uint4 *>(lo);
}

// ------------------------------------------------------------------ launchers
void split_bf16(const float *src, int rows, int K, __nv_bfloat16 *dst, cudaStream_t st) {
    const size_t n = (size_t)rows * (K / 8);
    if (n == 0) return;
    k_split_bf16<<<(int)((n + 255) / 256), 256, 0, st>>>(src, rows, K, dst);
    note_launches(1);
}

void pg_act1(int act, int Mp, int H, const float *Z, const float *b1, float *A1s, float *P1, float *Q1, float *Zd1,
             __nv_bfloat16 *hl, cudaStream_t st) {
    const int blocks = 148 * 8;
    if (act == 0) k_pg_act1<0><<<blocks, 256, 0, st>>>(Mp, H, Z, b1, A1s, P1, Q1, Zd1, hl);
    else k_pg_act1<1><<<blocks, 256, 0, st>>>(Mp, H, Z, b1, A1s, P1, Q1, Zd1, hl);
    note_launches(1);
}

void pg_act2(int act, int N, int Mp, int H, int B, const int32_t *atom_ptr, const int32_t *species, int S,
             const double *gE, const float *sigma, const float *w3, const float *b2, const float *b3, const float *Z,
             float *Zb2s, float *Y3, float *t_sig, float *t_c, float *t_cs, __nv_bfloat16 *hl, cudaStream_t st) {
    const int blocks = (Mp * 32 + 255) / 256;
    if (act == 0)
        k_pg_act2<0><<<blocks, 256, 0, st>>>(N, Mp, H, B, atom_ptr, species, S, gE, sigma, w3, b2, b3, Z, Zb2s, Y3,
                                             t_sig, t_c, t_cs, hl);
    else
        k_pg_act2<1><<<blocks, 256, 0, st>>>(N, Mp, H, B, atom_ptr, species, S, gE, sigma, w3, b2, b3, Z, Zb2s, Y3,
                                             t_sig, t_c, t_cs, hl);
    note_launches(1);
}

void pg_act1b(int Mp, int H, const float *Ab, const float *P1, const float *Q1, const float *Zd1, float *Zb1s,
              __nv_bfloat16 *hl, cudaStream_t st) {
    k_pg_act1b<<<148 * 8, 256, 0, st>>>(Mp, H, Ab, P1, Q1, Zd1, Zb1s, hl);
    note_launches(1);
}

void colsum3(int M, int H, const float *const A[3], float *const out[3], float *part, cudaStream_t st) {
    const int chunks = (M + CS_ROWS - 1) / CS_ROWS;
    ColSums cs;
    for (int a = 0; a < 3; ++a) {
        cs.A[a] = A[a];
        cs.out[a] = out[a];
    }
    if (chunks > 0) k_colsum_part<<<dim3((H + 31) / 32, chunks, 3), 256, 0, st>>>(M, H, cs, part);
    k_colsum_final<<<dim3((H + 31) / 32, 3), dim3(32, 8), 0, st>>>(chunks, H, cs, part);
    note_launches(chunks > 0 ? 2 : 1);
}

size_t colsum_part_floats(int M, int H) { return 3 * (size_t)((M + CS_ROWS - 1) / CS_ROWS) * H; }

// K slices of the weight gradient: enough 128 x 128 tile-slices for two blocks per SM, slices
// of at least 128 rows, at most 128 slices
int wgrad_ksplit(int K, int Mo, int No) {
    const int tiles = ((Mo + WG_T - 1) / WG_T) * ((No + WG_T - 1) / WG_T);
    int ks = (2 * 148 + tiles - 1) / tiles;
    const int kmax = K / 128;
    ks = ks > kmax ? kmax : ks;
    return ks < 1 ? 1 : (ks > 128 ? 128 : ks);
}

void wgrad(const float *A, int lda, const float *B, int ldb, int K, int Mo, int No, int Mstore, float *part, float *out,
           cudaStream_t st) {
    const int ks = wgrad_ksplit(K, Mo, No);
    int kchunk = (K + ks - 1) / ks;
    kchunk = (kchunk + WG_K - 1) / WG_K * WG_K;
    dim3 grid((Mo + WG_T - 1) / WG_T, (No + WG_T - 1) / WG_T, ks);
    k_wgrad<<<grid, 256, 0, st>>>(A, lda, B, ldb, K, Mo, No, kchunk, part);
    const size_t n = (size_t)Mstore * No;
    k_wgrad_reduce<<<(int)((n + WR_OUT - 1) / WR_OUT), dim3(WR_OUT, WR_GRP), 0, st>>>(ks, Mo, No, Mstore, part, out);
    note_launches(2);
}

size_t pg_tail_part_floats(int N, int S) { return (size_t)((N + TAIL_ATOMS - 1) / TAIL_ATOMS + 1) * (1 + 2 * S); }

void pg_tail(int N, const int32_t *species, int S, const float *t_sig, const float *t_c, const float *t_cs,
             float *part, float *g_sigma, float *g_mu, float *g_b3, cudaStream_t st) {
    const int nb = (N + TAIL_ATOMS - 1) / TAIL_ATOMS;
    if (nb > 0) k_pg_tail_part<<<nb, 256, 0, st>>>(N, species, S, t_sig, t_c, t_cs, part);
    k_pg_tail_final<<<1, ((1 + 2 * S + 31) / 32) * 32, 0, st>>>(nb, S, part, g_sigma, g_mu, g_b3);
    note_launches(nb > 0 ? 2 : 1);
}

void pg_beta_reduce(int nblocks, int nbeta, float scale, const float *part, float *out, cudaStream_t st) {
    k_pg_beta_reduce<<<(nbeta * 32 + 255) / 256, 256, 0, st>>>(nblocks, nbeta, scale, part, out);
    note_launches(1);
}

}  // namespace gm
