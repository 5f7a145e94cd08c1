// gm_gemm.h -- network GEMMs with fused epilogues (FP32 SIMT and BF16 tcgen05 paths).
//
// Every GEMM computes C[m][n] = sum_k A[m][k] * B[n][k]: A holds per-atom rows (M padded
// to a multiple of 128), B is a weight matrix stored with K contiguous.  The network of
// Eq. scale_shift runs as four of them per energy+forces evaluation:
//   L1  Z1 = G W1:        A1 = phi(Z1 + b1), D1 = phi'(Z1 + b1)
//   L2  Z2 = A1 W2:       a2 = phi(Z2 + b2); partial sums of a2 . w3 per 32 columns (energy);
//                         dZ2 = sigma_Z w3 phi'(Z2 + b2)          (dE_i/dZ2)
//   B1  dA1 = dZ2 W2^T:   dZ1 = dA1 * D1
//   B0  dG = dZ1 W1^T     (stored FP32)
// A shallow ensemble (E output heads, section "Uncertainty Quantification") runs L2 as
// EPI_L2E: w3 is the heads' mean (its gradient is the mean force) and the epilogue also
// writes each head's partial sums of a2 . w3e[k] per 32 columns.  Its per-head forces (the
// Jacobian mode, Eq. jacobian) need dZ2_k = sigma_Z w3e[k] phi'(Z2 + b2) for every head k;
// EPI_L2H writes those stacked rows from one L2 product (Z2 does not depend on the head).
#pragma once

#include "gm_internal.h"

namespace gm {

enum { EPI_L1 = 0, EPI_L2 = 1, EPI_B1 = 2, EPI_STORE = 3, EPI_L2E = 4, EPI_L2H = 5 };

struct EpiArgs {
    const float *bias;       // [N] (L1, L2)
    const float *w3;         // [N] (L2)
    const float *sigma;      // [S] (L2)
    const int32_t *species;  // [n_atoms] (L2)
    int n_atoms, n_species;
    void *out0;              // A1 (L1), dZ2 (L2), dZ1 (B1), C (STORE); row stride N
    void *out1;              // D1 (L1)
    const void *aux;         // D1 (B1)
    int aux_rows;            // B1: aux row = output row mod aux_rows (stacked heads), 0 = the row itself
    float *nn_part;          // [M][N/32] (L2): partial output-layer sums per 32 columns
    int n_ens;               // EPI_L2E: ensemble heads E
    const float *w3e;        // EPI_L2E: [E][N] head weights
    float *nn_ens;           // EPI_L2E: [E][N/32][nn_ens_ld] partial sums per head (rows minor)
    size_t nn_ens_ld;        // EPI_L2E: rows of nn_ens (>= M)
    int n_heads;             // EPI_L2H: heads whose dE/dz2 rows are written (w3 is [n_heads][N])
    size_t head_stride;      // EPI_L2H: output elements from one head's [M] rows to the next's
    int lo_out;              // BF16 outputs: also write the lo half (the consumer runs split)
    // Structure energies fused into the tcgen05 B1 GEMM (energy non-null; no virial): while
    // the first N tile of each row block runs its main loop, its four idle warps add E_i of
    // the block's rows (from nn_part, N/32 partials each) to the per-structure fixed-point
    // accumulators, and the last such block writes energy[] (gm_fixed.cuh)
    const int32_t *atom_ptr; // [n_structures + 1]
    int n_structures;
    const float *mu, *b3;    // [S], [1]
    unsigned long long *red_acc;
    double *energy;          // [n_structures]
    int debug_stall;         // tcgen05 path, tests of failure reporting: the producer issues no
                             // loads, so the MMA and epilogue waits run out (nothing in flight)
    int out_f16;             // tcgen05 L2/L2E/B1: write the output as FP16 in the hi slot of the
                             // [M][2N] layout (the FP16 backward GEMMs read it in one pass)
};
// BF16 operands of the tcgen05 path are stored as hi/lo pairs, [rows][2K]: columns [0, K)
// hold hi = bf16(x), columns [K, 2K) hold lo = bf16(x - hi).  A GEMM run with split = 0
// reads the hi half only; with split = 1 it accumulates hi*hi + lo*hi + hi*lo (three
// tensor-core passes, about FP32 accuracy).  The BF16 outputs of L1/L2/B1 are written in
// the same [M][2N] layout; D1 (phi') is kept in FP32.

// FP32 SIMT path (gm_gemm_simt.cu).  M % 128 == 0, N % 64 == 0, K % 16 == 0.
void gemm_f32(int epi, int act, const float *A, const float *B, int M, int N, int K, const EpiArgs &e,
              cudaStream_t st);

// BF16 tcgen05 path (gm_gemm_tc.cu).  M % 128 == 0, N % 64 == 0, K % 64 == 0; A [M][2K] and
// B [N][2K] BF16 hi/lo pairs with 16-byte aligned rows.  L1/L2/B1 outputs are BF16 hi/lo
// pairs [M][2N] (D1 FP32 [M][N]), STORE is FP32 [M][N].
// forced_bn = 0 picks the tile width from the problem size (64, 128 or 256 columns).
// forced_cps = 0 picks one or two CTAs per SM from the tile count (two halve the stage ring
// and overlap one CTA's epilogue with the other's main loop).
// f16 = 1: A and B hold FP16 (not BF16) in their hi slots, read in one pass (split must be 0;
// one MMA always takes both operands in the same type)
gm_status gemm_bf16(int epi, int act, const __nv_bfloat16 *A, const __nv_bfloat16 *B, int M, int N, int K, int split,
                    const EpiArgs &e, int32_t *status, cudaStream_t st, int forced_bn = 0, int forced_cps = 0,
                    int f16 = 0);
int tc_choose_bn(int M, int N, int forced);

// The mixed path's whole network in one tcgen05 kernel per 128-row tile (gm_mlp_fused.cuh):
// L1 and L2 on BF16 operands (single pass), B1 and B0 on FP16 operands; a1, dZ2 and dZ1 stay
// in shared memory.  G [M][2 NFP] BF16 (hi slots), W1t [H][2 NFP], W2t [H][2H] BF16,
// W2 [H][2H], W1p [NFP][2H] FP16 (hi slots).  Outputs: D1 [M][H] FP16 (phi'(z1)), nn_part
// [M][H/32], dG [M][NFP] FP32.  H must be 128, 256 or 512.
struct FusedMlpArgs {
    int n_atoms, n_species;
    const int32_t *species;
    const float *b1, *b2, *w3, *sigma;
    __half *D1;               // [M][H] FP16 phi'(z1) (scratch)
    float *nn_part, *dG;
    int debug_stall = 0;      // failure-reporting tests: no operand loads, every wait runs out
    int ctas = 0;             // per-tile kernel: CTAs of the persistent launch (0: one per SM)
    // cluster kernel only: [M][2H] scratch arrays through which the cluster gathers a1, dZ2
    // and dZ1 (first H columns), and the structure energies summed in the kernel (energy
    // null: not summed)
    __nv_bfloat16 *xa1 = nullptr, *xdz2 = nullptr, *xdz1 = nullptr;
    const int32_t *atom_ptr = nullptr;
    int n_structures = 0;
    const float *mu = nullptr, *b3 = nullptr;
    unsigned long long *red_acc = nullptr;
    double *energy = nullptr;
};
bool mlp_fused_supported(int H);
gm_status mlp_fused(int act, int M, int H, const __nv_bfloat16 *G, const __nv_bfloat16 *W1t, const __nv_bfloat16 *W2t,
                    const __half *W2, const __half *W1p, const FusedMlpArgs &a, int32_t *status, cudaStream_t st);

// The same network with each 128-row tile split over a cluster of cs CTAs along the hidden
// width (gm_mlp_cluster.cuh): cs in 2, 4, 8 with H / cs >= 64.  When a.energy is set the
// structure energies are summed in the kernel (into a.red_acc, fixed point) and written to
// a.energy.  mlp_cluster_capacity: clusters the device keeps resident at once (0: the
// configuration cannot launch, or is not supported).
bool mlp_cluster_supported(int H, int cs);
int mlp_cluster_capacity(int act, int H, int cs);
gm_status mlp_cluster(int act, int M, int H, int cs, const __nv_bfloat16 *G, const __nv_bfloat16 *W1t,
                      const __nv_bfloat16 *W2t, const __half *W2, const __half *W1p, const FusedMlpArgs &a,
                      int32_t *status, cudaStream_t st);

}  // namespace gm
