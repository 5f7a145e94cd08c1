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
// Kernel attributes (cudaFuncSetAttribute) belong to the current device: a launcher keeps one
// flag per device and sets them the first time it launches on that device.
struct PerDeviceOnce {
    bool done[64] = {};
    bool first() {
        int d = 0;
        if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return true;
        if (done[d]) return false;
        done[d] = true;
        return true;
    }
};

// SM count of the current device (cached per device)
int device_sm_count();

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


// ---- tracing (gm_api.cu): kernel-launch counter and stage timing
enum Stage {
    ST_NEIGHBORS = 0, ST_MOMENTS, ST_CONTRACT_FWD, ST_GEMM_L1, ST_GEMM_L2, ST_GEMM_B1, ST_GEMM_B0,
    ST_CONTRACT_BWD, ST_FORCES, ST_REDUCE, ST_PG_PAIR_FWD, ST_PG_NETWORK, ST_PG_PAIR_BWD, ST_NL_BIN, ST_NL_COUNT,
    ST_NL_SCAN, ST_NL_FILL, ST_NL_COOP, ST_MD, ST_MLP_FUSED, N_STAGES
};
void note_launches(int n);

// Programmatic dependent launch: the kernel may be scheduled while its predecessor on the
// stream drains (its launch latency and any independent prologue overlap the predecessor's
// tail).  Every kernel launched this way calls griddep_wait() before it reads or writes
// global memory that earlier kernels of the stream use; the wait returns once those kernels
// have completed and their writes are visible (and at once when there is no predecessor).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

struct StageScope {
    int stage;
    cudaStream_t st;
    void *ev0;
    bool in_graph;
    StageScope(int s, cudaStream_t stream);
    ~StageScope();
};

// ---- model and error accessors, argument checks (gm_api.cu)
const gm_model_desc *model_desc(const gm_model *m);
gm_status set_last_error(gm_status s, const char *msg);
// GM_ERR_ARG / GM_ERR_UNSUPPORTED (with gm_last_error set) for a system or neighbour list
// that no kernel may be launched on: null or misaligned pointers, bad sizes
gm_status check_system(const gm_model *m, const gm_system *s);
gm_status check_nlist(const gm_system *s, const gm_nlist *nl, bool need_pairs);
// GM_ERR_CUDA (with the runtime's message) if a launch of this thread failed, else GM_OK
gm_status launch_status();
// GM_ERR_ARG unless `stream` belongs to the current device
gm_status check_stream_device(cudaStream_t stream);

// ---- neighbour search (gm_nlist.cu)
struct NlTuning {
    int mode = GM_NL_MODE_AUTO;   // GM_NL_MODE_* of gm.h
    int split = 0;                // blocks per home cell in the search passes (0 = by size)
    int blocks = 0;               // blocks of the cooperative launch (0 = by size)
    int two_pass = 0;             // 1: count and fill passes even when the workspace holds the slab
    int items = 0;                // search work items: 0 = by size, 1 = per block, 2 = per warp, 3 = brute force
    int debug_stall = 0;          // 1: block 0 of the cooperative build skips the grid barriers (tests)
};
const NlTuning &nl_tuning(const gm_model *m);
size_t nl_workspace_bytes(int n_struct, int n_atoms, int64_t capacity);   // with the search slab
size_t nl_workspace_min_bytes(int n_struct, int n_atoms);                  // two-pass search
// gate (device int32, may be null): build only when *gate != 0 at launch; the list is left as
// it was otherwise (the memset of the build's own counters still runs)
gm_status nl_build(const gm_system &sys, double r_cut, int n_species, gm_nlist &nl, void *ws, size_t ws_bytes,
                   int32_t *status, cudaStream_t st, const NlTuning &tune, const int32_t *gate = nullptr);

}  // namespace gm
