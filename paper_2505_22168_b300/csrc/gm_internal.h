// gm_internal.h -- declarations shared by the libgm translation units (not public).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stddef.h>
#include <stdint.h>

#include "gm.h"
#include "gm_common.cuh"

namespace gm {

// Bump allocator over the caller's workspace (256-byte aligned slices).
struct Carve {
    char *base;
    size_t off, cap;
    bool ok = true;
    Carve(void *b, size_t c) : base(static_cast<char *>(b)), off(0), cap(c) {}
    template <class T>
    T *take(size_t n) {
        size_t start = (off + 255) & ~size_t(255);
        size_t bytes = n * sizeof(T);
        off = start + bytes;
        if (off > cap || base == nullptr) { ok = false; return nullptr; }
        return reinterpret_cast<T *>(base + start);
    }
};

// Per-structure cell-list geometry (device, in the neighbour workspace).
struct NlStruct {
    double L[3];     // orthorhombic box edges
    double cs[3];    // cell edge per axis (>= r_cut unless the box is smaller)
    int nc[3];       // cells per axis
    int K[3];        // stencil half-width per axis (cells)
    int cell0;       // first global cell index of this structure
    int a0, n;       // atoms
    float Lf[3];     // edges in FP32 (distance filter)
    float eps2;      // half-width of the FP32 band around r_cut^2 decided in FP64
};

// ---- tracing (gm_api.cu): kernel-launch counter and stage timing
enum Stage {
    ST_NEIGHBORS = 0, ST_MOMENTS, ST_CONTRACT_FWD, ST_GEMM_L1, ST_GEMM_L2, ST_GEMM_B1, ST_GEMM_B0,
    ST_CONTRACT_BWD, ST_FORCES, ST_REDUCE, ST_PG_PAIR_FWD, ST_PG_NETWORK, ST_PG_PAIR_BWD, ST_NL_BIN, ST_NL_COUNT,
    ST_NL_SCAN, ST_NL_FILL, N_STAGES
};
void note_launches(int n);
struct StageScope {
    int stage;
    cudaStream_t st;
    void *ev0;
    bool in_graph;
    StageScope(int s, cudaStream_t stream);
    ~StageScope();
};

// ---- model and error accessors (gm_api.cu)
const gm_model_desc *model_desc(const gm_model *m);
gm_status set_last_error(gm_status s, const char *msg);

// ---- neighbour search (gm_nlist.cu)
size_t nl_workspace_bytes(int n_struct, int n_atoms);
gm_status nl_build(const gm_system &sys, double r_cut, int n_species, gm_nlist &nl, void *ws, size_t ws_bytes,
                   int32_t *status, cudaStream_t st);

// ---- device-wide exclusive scan (gm_nlist.cu): out[0..n] with out[n] = total
size_t scan_tmp_ints(int n);
void exclusive_scan(const int32_t *in, int32_t *out, int n, int32_t *tmp, cudaStream_t st);

}  // namespace gm
