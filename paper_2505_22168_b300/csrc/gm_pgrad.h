// gm_pgrad.h -- launchers of the network part of the parameter gradient (gm_pgrad.cu).
#pragma once

#include "gm_internal.h"

namespace gm {

// hl (mixed path; null in the FP32 path): the kernel also writes the hi/lo BF16 rows of the
// stacked array it produces (A1s, Zb2s, Zb1s), the next GEMM's A operand
void pg_act1(int act, int Mp, int H, const float *Z, const float *b1, float *A1s, float *P1, float *Q1, float *Zd1,
             __nv_bfloat16 *hl, cudaStream_t st);
void pg_act2(int act, int N, int Mp, int H, int B, const int32_t *atom_ptr, const int32_t *species, int S,
             const double *gE, const float *sigma, const float *w3, const float *b2, const float *b3, const float *Z,
             float *Zb2s, float *Y3, float *t_sig, float *t_c, float *t_cs, __nv_bfloat16 *hl, cudaStream_t st);
void pg_act1b(int Mp, int H, const float *Ab, const float *P1, const float *Q1, const float *Zd1, float *Zb1s,
              __nv_bfloat16 *hl, cudaStream_t st);
// out[a][h] = sum_{m < M} A[a][m][h] for three arrays [M][H]; part holds colsum_part_floats(M, H)
void colsum3(int M, int H, const float *const A[3], float *const out[3], float *part, cudaStream_t st);
size_t colsum_part_floats(int M, int H);
int wgrad_ksplit(int K, int Mo, int No);
// out[i][j] (i < Mstore) = sum_k A[k][i] B[k][j], A [K][lda], B [K][ldb]; part holds ksplit x Mo x No
void wgrad(const float *A, int lda, const float *B, int ldb, int K, int Mo, int No, int Mstore, float *part, float *out,
           cudaStream_t st);
// part holds pg_tail_part_floats(N, S) floats
void pg_tail(int N, const int32_t *species, int S, const float *t_sig, const float *t_c, const float *t_cs,
             float *part, float *g_sigma, float *g_mu, float *g_b3, cudaStream_t st);
size_t pg_tail_part_floats(int N, int S);
void pg_beta_reduce(int nblocks, int nbeta, float scale, const float *part, float *out, cudaStream_t st);
// hi/lo BF16 copy of src [rows][K] (K a multiple of 8): dst [rows][2K]
void split_bf16(const float *src, int rows, int K, __nv_bfloat16 *dst, cudaStream_t st);

}  // namespace gm
