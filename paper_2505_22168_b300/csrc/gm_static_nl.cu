// gm_static_nl.cu -- neighbour build that allocates nothing and takes no workspace.
//
// For callers that cannot allocate device memory themselves: a host program that has
// handed all device memory to its own pool (an MD engine embedding this library), or a
// time-stepping loop that must not call cudaMalloc, whose implicit synchronisation
// would stall every other stream in the middle of a step.  gm_build_neighbors needs a
// caller-provided workspace; this variant uses a fixed array in the library's own
// device memory instead.
//
// The array is a file-scope __device__ variable of GM_NOALLOC_SCRATCH_BYTES bytes.  Every
// GPU that loads the library holds it until the process exits.  Host code cannot use the
// variable's name as a device address, so the first call on each device (with that
// device current) looks its address up with cudaGetSymbolAddress and caches it.  All
// calls share the array: it keeps the previous call's contents (the build clears what
// must start at zero), and calls that overlap on the GPU -- on different streams, or
// from different threads -- race on it.
#include <mutex>

#include "gm_internal.h"

namespace {

constexpr size_t GM_NOALLOC_SCRATCH_BYTES = size_t(8) << 20;  // 8 MiB
constexpr int GM_NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_nl_scratch[GM_NOALLOC_SCRATCH_BYTES];

std::mutex g_scratch_mu;
void *g_scratch_ptr[GM_NOALLOC_MAX_DEVICES] = {};

gm_status scratch_address(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= GM_NOALLOC_MAX_DEVICES) return GM_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (g_scratch_ptr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_nl_scratch) != cudaSuccess || p == nullptr) return GM_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return GM_OK;
}

}  // namespace

extern "C" {

gm_status gm_build_neighbors_noalloc(const gm_model *m, const gm_system *sys, gm_nlist *nl, int32_t *status_dev,
                                     struct CUstream_st *stream) {
    using gm::set_last_error;
    // the same argument checks as gm_build_neighbors: nothing is launched on a null or
    // misaligned pointer
    gm_status s = gm::check_system(m, sys);
    if (s != GM_OK) return s;
    if ((s = gm::check_nlist(sys, nl, false)) != GM_OK) return s;
    if (!status_dev) return set_last_error(GM_ERR_ARG, "null status");
    // the cached scratch address is the current device's, so the stream must be too
    if ((s = gm::check_stream_device(stream)) != GM_OK) return s;
    const size_t need = gm::nl_workspace_min_bytes(sys->n_structures, sys->n_atoms);
    if (need > GM_NOALLOC_SCRATCH_BYTES)
        return set_last_error(GM_ERR_WORKSPACE,
                              "system too large for the fixed 8 MiB scratch of gm_build_neighbors_noalloc "
                              "(its minimum neighbour workspace exceeds 8 MiB: about 90,000 atoms in one "
                              "structure); use gm_build_neighbors with a workspace");
    void *scratch = nullptr;
    if (scratch_address(&scratch) != GM_OK)
        return set_last_error(GM_ERR_CUDA, "cudaGetSymbolAddress of the fixed scratch failed");
    const gm_model_desc *d = gm::model_desc(m);
    {
        gm::StageScope sc(gm::ST_NEIGHBORS, stream);
        s = gm::nl_build(*sys, d->r_cut, d->n_species, *nl, scratch, GM_NOALLOC_SCRATCH_BYTES, status_dev, stream,
                         gm::nl_tuning(m));
    }
    if (s != GM_OK) return set_last_error(s, "neighbour build launch failed");
    return gm::launch_status();
}

}  // extern "C"
