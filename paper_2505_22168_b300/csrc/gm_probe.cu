// gm_probe.cu -- throughput probes that give the roofline denominators of the FP32 kernels.
//
// The pair kernels and contractions are bound by FP32 fused multiply-adds and by the
// special-function unit (exp2, sin/cos).  These kernels issue nothing but long independent
// chains of one operation on every SM, so CUDA-event time over a launch gives the device's
// sustained rate for that operation: the peak a kernel of the library is compared with.
#include "gm_internal.h"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;   // independent dependency chains per thread

// FFMA: every iteration issues PROBE_CHAINS x 8 FMAs (2 flop each) per thread.
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_ffma(int64_t iters, float *sink) {
    float a[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) a[c] = 1e-3f * (threadIdx.x + c);
    const float b = 0.9999f, d = 1e-6f;
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int c = 0; c < PROBE_CHAINS; ++c) a[c] = fmaf(a[c], b, d);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) s += a[c];
    if (s == 123456.0f) sink[blockIdx.x] = s;   // never true; keeps the chains live
}

// MUFU: every iteration issues PROBE_CHAINS x 8 base-2 exponentials per thread (ex2.approx,
// the instruction behind the radial Gaussians), with one FMA each to keep the argument bounded.
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_mufu(int64_t iters, float *sink) {
    float a[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) a[c] = -1e-3f * (threadIdx.x + c);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int c = 0; c < PROBE_CHAINS; ++c) a[c] = ex2_approx(a[c]) - 1.0f;
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) s += a[c];
    if (s == 123456.0f) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" gm_status gm_probe_alu(int32_t kind, int64_t iters, float *sink, double *ops, struct CUstream_st *stream) {
    if (kind < 0 || kind > 1 || iters < 1 || !sink || !ops) return gm::set_last_error(GM_ERR_ARG, "bad probe argument");
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return gm::set_last_error(GM_ERR_CUDA, "device query failed");
    void (*kern)(int64_t, float *) = kind == 0 ? k_probe_ffma : k_probe_mufu;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PROBE_THREADS, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int blocks = sms * per_sm;
    kern<<<blocks, PROBE_THREADS, 0, stream>>>(iters, sink);
    gm::note_launches(1);
    // FFMA: 2 flop per FMA; MUFU: one exponential per operation (the FMA beside it not counted)
    const double per_iter = (double)PROBE_CHAINS * 8.0 * (kind == 0 ? 2.0 : 1.0);
    *ops = per_iter * (double)iters * (double)blocks * PROBE_THREADS;
    return gm::launch_status();
}
