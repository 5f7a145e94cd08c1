// gm_contract.h -- launchers of the contraction kernels (Eq. contraction).
#pragma once

#include "gm_internal.h"

namespace gm {

// psi [N][100] FP32 -> G [Mp][384] FP32, or G [Mp][2*384] BF16 hi/lo pairs (rows >= N and
// feature columns >= 360 zero).
// features_out [N][360] FP32 (optional copy for diagnostics, may be NULL).
void launch_contract_fwd_f32(const float *psi, int N, int Mp, float *G, float *features_out, cudaStream_t st);
// lo_out: also write the lo halves of the hi/lo BF16 rows (needed when the first network
// GEMM runs with the split passes)
void launch_contract_fwd_bf16(const float *psi, int N, int Mp, __nv_bfloat16 *G, float *features_out, bool lo_out,
                              cudaStream_t st);
// dE/dG [Mp][384] FP32 and psi -> dE/dpsi [N][100] FP32 (unique components)
// dg_tiled: dG in the per-tile fused network kernel's layout (per 128-row tile, 4-column groups
// major and rows minor), else row-major [Mp][384].  heads > 1: the dE/dG of that many
// shallow-ensemble heads, dg_head_stride floats apart, into dpsi [heads][N][100] in one launch
void launch_contract_bwd(const float *psi, const float *dG, int N, float *dpsi, cudaStream_t st,
                         bool dg_tiled = false, int heads = 1, size_t dg_head_stride = 0);

// Parameter gradient: GG [2Mp][384] = [G; dG/dPsi . psid]; and from Gbs = [dJ/dG; dJ/dGd]
// the moment adjoints psib, psidb [N][100] (see gm_contract.cu).
void launch_contract_fwd_dual(const float *psi, const float *psid, int N, int Mp, float *GG, cudaStream_t st);
void launch_contract_bwd_dual(const float *psi, const float *psid, const float *Gbs, int N, int Mp, float *psib,
                              float *psidb, cudaStream_t st);

}  // namespace gm
