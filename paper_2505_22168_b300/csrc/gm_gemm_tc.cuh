// gm_gemm_tc.cuh -- BF16 network GEMM on the 5th-generation tensor cores (tcgen05), sm_103a.
//
// C[m][n] = sum_k A[m][k] B[n][k] with A, B BF16 (K contiguous), FP32 accumulation in TMEM,
// and the epilogues of gm_gemm.h.  One CTA computes a 128 x BN tile:
//   warp 0 lane 0  TMA producer: 64-wide K blocks of A (128 rows) and B (BN rows) into a
//                  STAGES-deep shared-memory ring (128-byte swizzle), mbarrier complete_tx
//   warp 1 lane 0  MMA issuer: 4 x tcgen05.mma (M=128, N=BN, K=16) per K block into one
//                  TMEM accumulator; tcgen05.commit frees the stage, a final commit
//                  signals the epilogue
//   warps 0..7     epilogue: tcgen05.ld 32 lanes x 32 columns per chunk (thread = row;
//                  warps w and w + 4 share TMEM lanes and split the columns)
// Every wait on an mbarrier is bounded (about one second of %globaltimer); on expiry the
// kernel records GM_ERR_TIMEOUT in the status word, waits (bounded) for the copies it
// issued, releases its TMEM and returns.
#pragma once

#include <cuda.h>

#include "gm_fixed.cuh"
#include "gm_gemm.h"

namespace gm {
namespace tc {

constexpr int BM = 128;
constexpr int BK = 64;                      // BF16 elements per 128-byte swizzle row
constexpr int A_STAGE_BYTES = BM * BK * 2;  // 16 KiB
constexpr uint64_t WAIT_NS = 1000000000ull; // bound of every wait

// stage ring: about 192 KB for one CTA per SM, about 96 KB when two CTAs share an SM (one
// CTA's epilogue then overlaps the other's main loop)
__host__ __device__ constexpr int stages_for(int bn, int cps = 1) {
    return cps == 1 ? (bn >= 256 ? 4 : 6) : (bn >= 256 ? 2 : (bn >= 128 ? 3 : 4));
}
__host__ __device__ constexpr int tmem_cols_for(int bn) { return bn <= 32 ? 32 : (bn <= 64 ? 64 : (bn <= 128 ? 128 : 256)); }
__host__ __device__ constexpr size_t ring_bytes_for(int bn, int cps = 1) {
    return (size_t)stages_for(bn, cps) * (A_STAGE_BYTES + bn * BK * 2);
}
__host__ __device__ constexpr size_t smem_bytes_for(int bn, int cps = 1) {
    return ring_bytes_for(bn, cps) + 1024 + 256;
}

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of the given parity; false on timeout or abort.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = now_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (now_ns() - t0 > WAIT_NS) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int c_inner, int c_row) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            su32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(su32(bar)), "r"(c_inner), "r"(c_row)
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, M = 128, N = bn.
__host__ __device__ constexpr uint32_t instr_desc(int bn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}
// the same with A and B FP16 (format code 0 in both operand fields)
__host__ __device__ constexpr uint32_t instr_desc_f16(int bn) {
    return (1u << 4) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

// 32 TMEM lanes x 32 consecutive 32-bit columns; thread t of the warp gets lane (base + t).
__device__ __forceinline__ void tmem_ld_32cols(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ uint4 pack8_bf16(const float *x) {
    uint4 o;
    __nv_bfloat162 h0 = __floats2bfloat162_rn(x[0], x[1]), h1 = __floats2bfloat162_rn(x[2], x[3]);
    __nv_bfloat162 h2 = __floats2bfloat162_rn(x[4], x[5]), h3 = __floats2bfloat162_rn(x[6], x[7]);
    o.x = *reinterpret_cast<uint32_t *>(&h0);
    o.y = *reinterpret_cast<uint32_t *>(&h1);
    o.z = *reinterpret_cast<uint32_t *>(&h2);
    o.w = *reinterpret_cast<uint32_t *>(&h3);
    return o;
}

// hi/lo split of 8 values: hi = bf16(x), lo = bf16(x - hi)
__device__ __forceinline__ void pack8_split(const float *x, uint4 &hi, uint4 &lo) {
    float h[8], l[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        h[t] = __bfloat162float(__float2bfloat16_rn(x[t]));
        l[t] = x[t] - h[t];
    }
    hi = pack8_bf16(h);
    lo = pack8_bf16(l);
}

__device__ __forceinline__ uint4 pack8_f16(const float *x) {
    uint4 o;
    __half2 h0 = __floats2half2_rn(x[0], x[1]), h1 = __floats2half2_rn(x[2], x[3]);
    __half2 h2 = __floats2half2_rn(x[4], x[5]), h3 = __floats2half2_rn(x[6], x[7]);
    o.x = *reinterpret_cast<uint32_t *>(&h0);
    o.y = *reinterpret_cast<uint32_t *>(&h1);
    o.z = *reinterpret_cast<uint32_t *>(&h2);
    o.w = *reinterpret_cast<uint32_t *>(&h3);
    return o;
}

__device__ __forceinline__ void unpack8_bf16(uint4 u, float *x) {
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float2 f = __bfloat1622float2(h[q]);
        x[2 * q] = f.x;
        x[2 * q + 1] = f.y;
    }
}

// Activation for the BF16 path: SiLU with the fast exponential and division (their
// error is far below BF16 rounding); tanh stays accurate (its derivative gates forces).
template <int ACT>
__device__ __forceinline__ float act_fast(float z, float &d1) {
    if (ACT == 0) return act_fwd<0>(z, d1);
    const float s = __fdividef(1.0f, 1.0f + __expf(-z));
    d1 = s * (1.0f + z * (1.0f - s));
    return z * s;
}

// Per-warp staging of a 32-row x 32-column tile in the (then idle) stage ring, so that rows
// held one per thread leave and arrive as whole 64- or 128-byte row segments: rows padded to
// 80 and 144 bytes keep the 16-byte accesses of a warp on distinct banks.
struct EpiStage {
    uint4 hi[32][5];
    uint4 lo[32][5];
    float4 d[32][9];
};
constexpr size_t EPI_STAGE_BYTES = sizeof(EpiStage);

// 32 rows x 32 BF16 (64 B a row) from the staging rows to out[row0 + r][col0 ..]
__device__ __forceinline__ void warp_store_bf16(const uint4 (*st)[5], __nv_bfloat16 *out, int row0, size_t ld,
                                                int col0, int lane) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int idx = i * 32 + lane, r = idx >> 2, q = idx & 3;
        *reinterpret_cast<uint4 *>(out + (size_t)(row0 + r) * ld + col0 + q * 8) = st[r][q];
    }
}
// 32 rows x 32 FP32 (128 B a row), staging to global and global to staging
__device__ __forceinline__ void warp_store_f32(const float4 (*st)[9], float *out, int row0, size_t ld, int col0,
                                               int lane) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int idx = i * 32 + lane, r = idx >> 3, q = idx & 7;
        *reinterpret_cast<float4 *>(out + (size_t)(row0 + r) * ld + col0 + q * 4) = st[r][q];
    }
}
__device__ __forceinline__ void warp_load_f32(float4 (*st)[9], const float *in, int row0, size_t ld, int col0,
                                              int lane) {
    float4 t[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int idx = i * 32 + lane, r = idx >> 3, q = idx & 7;
        t[i] = __ldg(reinterpret_cast<const float4 *>(in + (size_t)(row0 + r) * ld + col0 + q * 4));
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int idx = i * 32 + lane, r = idx >> 3, q = idx & 7;
        st[r][q] = t[i];
    }
}

// Epilogue of one row segment of 32 columns starting at column n (multiple of 32); the warp's
// 32 rows start at row0 and this thread holds row row0 + lane.  BF16 outputs go to [m][n]
// (hi) and, when e.lo_out, [m][N + n] (lo) of a [M][2N] array.
template <int EPI, int ACT>
__device__ __forceinline__ void epilogue32(const EpiArgs &e, int row0, int n, int N, float (&v)[32], float &part,
                                           EpiStage &sg, int lane) {
    const int m = row0 + lane;
    if (EPI == EPI_L2H) {
        // y = sigma_Z phi'(Z2 + b2) once, then one [M][2N] block of rows per head
        const float sg_m = m < e.n_atoms ? e.sigma[min(max(e.species[m], 0), e.n_species - 1)] : 0.0f;
        float y[32];
#pragma unroll
        for (int t = 0; t < 32; ++t) {
            float d;
            act_fast<ACT>(v[t] + __ldg(e.bias + n + t), d);
            y[t] = sg_m * d;
        }
        __nv_bfloat16 *ob = static_cast<__nv_bfloat16 *>(e.out0);
#pragma unroll 1
        for (int k = 0; k < e.n_heads; ++k, ob += e.head_stride) {
            const float *wk = e.w3 + (size_t)k * N + n;
            float yk[32];
#pragma unroll
            for (int t = 0; t < 32; ++t) yk[t] = y[t] * __ldg(wk + t);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (e.out_f16) {
                    sg.hi[lane][q] = pack8_f16(yk + 8 * q);
                } else {
                    uint4 hi, lo;
                    pack8_split(yk + 8 * q, hi, lo);
                    sg.hi[lane][q] = hi;
                    sg.lo[lane][q] = lo;
                }
            }
            __syncwarp();
            warp_store_bf16(sg.hi, ob, row0, 2 * (size_t)N, n, lane);
            if (e.lo_out && !e.out_f16) warp_store_bf16(sg.lo, ob + N, row0, 2 * (size_t)N, n, lane);
            __syncwarp();
        }
        return;
    }
    if (EPI == EPI_STORE) {
#pragma unroll
        for (int q = 0; q < 8; ++q) sg.d[lane][q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        __syncwarp();
        warp_store_f32(sg.d, static_cast<float *>(e.out0), row0, N, n, lane);
        __syncwarp();
        return;
    }
    float y[32];
    if (EPI == EPI_B1) {
        warp_load_f32(sg.d, static_cast<const float *>(e.aux), e.aux_rows ? row0 % e.aux_rows : row0, N, n, lane);
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float4 g = sg.d[lane][q];
            y[4 * q] = v[4 * q] * g.x;
            y[4 * q + 1] = v[4 * q + 1] * g.y;
            y[4 * q + 2] = v[4 * q + 2] * g.z;
            y[4 * q + 3] = v[4 * q + 3] * g.w;
        }
    } else if (EPI == EPI_L1) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            float d[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) y[4 * q + t] = act_fast<ACT>(v[4 * q + t] + __ldg(e.bias + n + 4 * q + t), d[t]);
            sg.d[lane][q] = make_float4(d[0], d[1], d[2], d[3]);
        }
    } else {  // EPI_L2, EPI_L2E
        const float sg_m = m < e.n_atoms ? e.sigma[min(max(e.species[m], 0), e.n_species - 1)] : 0.0f;
        float av[32];
#pragma unroll
        for (int t = 0; t < 32; ++t) {
            float d;
            const int c = n + t;
            const float a = act_fast<ACT>(v[t] + __ldg(e.bias + c), d);
            const float w = __ldg(e.w3 + c);
            part = fmaf(a, w, part);
            y[t] = sg_m * w * d;
            av[t] = a;
        }
        if (EPI == EPI_L2E) {
            for (int k = 0; k < e.n_ens; ++k) {
                // head k's 32 weights of this chunk: eight 16-byte loads, the same for every lane
                const float4 *wk = reinterpret_cast<const float4 *>(e.w3e + (size_t)k * N + n);
                float p = 0.0f;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float4 w = __ldg(wk + q);
                    p = fmaf(av[4 * q], w.x, p);
                    p = fmaf(av[4 * q + 1], w.y, p);
                    p = fmaf(av[4 * q + 2], w.z, p);
                    p = fmaf(av[4 * q + 3], w.w, p);
                }
                e.nn_ens[((size_t)k * (N / 32) + n / 32) * e.nn_ens_ld + m] = p;
            }
        }
    }
    const bool f16 = EPI != EPI_L1 && e.out_f16;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (f16) {
            sg.hi[lane][q] = pack8_f16(y + 8 * q);
        } else {
            uint4 hi, lo;
            pack8_split(y + 8 * q, hi, lo);
            sg.hi[lane][q] = hi;
            sg.lo[lane][q] = lo;
        }
    }
    __syncwarp();
    __nv_bfloat16 *ob = static_cast<__nv_bfloat16 *>(e.out0);
    warp_store_bf16(sg.hi, ob, row0, 2 * (size_t)N, n, lane);
    if (e.lo_out && !f16) warp_store_bf16(sg.lo, ob + N, row0, 2 * (size_t)N, n, lane);
    if (EPI == EPI_L1) warp_store_f32(sg.d, static_cast<float *>(e.out1), row0, N, n, lane);
    __syncwarp();
}

static_assert(8 * sizeof(EpiStage) <= ring_bytes_for(64, 2) && 8 * sizeof(EpiStage) <= ring_bytes_for(256, 2),
              "epilogue staging must fit in the stage ring");

template <int BN, int EPI, int ACT, int CPS>
__global__ void __launch_bounds__(256, CPS)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N, int K,
              int split, EpiArgs e, int32_t *status, int f16) {
    constexpr int STAGES = stages_for(BN, CPS);
    constexpr int B_STAGE_BYTES = BN * BK * 2;
    constexpr int STAGE_BYTES = A_STAGE_BYTES + B_STAGE_BYTES;
    constexpr uint32_t TMEM_COLS = tmem_cols_for(BN);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *done = empty + STAGES;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the N tiles of one row block are consecutive blocks, so the A rows come from DRAM once
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int KB1 = K / BK;                 // K blocks of one pass
    // Split operands (hi | lo halves along K): with a ring of at least four stages, stage
    // pairs hold the four tiles of one K block (A hi, B hi, A lo, B lo) and the three products
    // hi*hi, lo*hi, hi*lo run on them (each tile loaded once); otherwise three passes over K
    // (hi*hi, lo*hi, hi*lo), the hi tiles loaded twice.
    constexpr bool FUSED_OK = STAGES >= 4;
    const bool fused = split && FUSED_OK;
    constexpr int FST = STAGES / 2;         // fused stages (pairs of ring stages)
    const int KB = split ? (fused ? KB1 : 3 * KB1) : KB1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        tmem_alloc(tmem_slot, TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    griddep_wait();                         // operands and epilogue inputs come from earlier kernels

    // tests of failure reporting: a producer that issues nothing (no copy is ever in flight)
    const int KB_LOAD = e.debug_stall ? 0 : KB;
    if (warp == 0 && lane == 0 && fused) {
        // ---------------- TMA producer, fused split: one stage pair per K block
        int issued = 0;
        for (int kb = 0; kb < KB_LOAD; ++kb) {
            const int s = kb % FST;
            if (kb >= FST && !mbar_wait(empty + s, ((kb / FST) - 1) & 1, abort_flag)) {
                *abort_flag = 1;
                break;
            }
            uint8_t *hi_dst = smem + (2 * s) * STAGE_BYTES;
            uint8_t *lo_dst = hi_dst + STAGE_BYTES;
            mbar_expect_tx(full + s, 2 * STAGE_BYTES);
            tma_load_2d(hi_dst, &tmA, full + s, kb * BK, m0);
            tma_load_2d(hi_dst + A_STAGE_BYTES, &tmB, full + s, kb * BK, n0);
            tma_load_2d(lo_dst, &tmA, full + s, K + kb * BK, m0);
            tma_load_2d(lo_dst + A_STAGE_BYTES, &tmB, full + s, K + kb * BK, n0);
            ++issued;
        }
        if (*abort_flag) {
            for (int kb = (issued > FST ? issued - FST : 0); kb < issued; ++kb) {
                volatile int never = 0;
                mbar_wait(full + (kb % FST), (kb / FST) & 1, &never);
            }
        }
    } else if (warp == 1 && lane == 0 && fused) {
        // ---------------- MMA issuer, fused split
        const uint32_t idesc = f16 ? instr_desc_f16(BN) : instr_desc(BN);
        bool ok = true;
        for (int kb = 0; kb < KB; ++kb) {
            const int s = kb % FST;
            if (!mbar_wait(full + s, (kb / FST) & 1, abort_flag)) {
                *abort_flag = 1;
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t ah = su32(smem + (2 * s) * STAGE_BYTES), bh = ah + A_STAGE_BYTES;
            const uint32_t al = ah + STAGE_BYTES, bl = al + A_STAGE_BYTES;
#pragma unroll
            for (int k = 0; k < BK / 16; ++k) {
                umma_bf16(tmem, smem_desc(ah + 32 * k), smem_desc(bh + 32 * k), idesc, (kb | k) != 0);
                umma_bf16(tmem, smem_desc(al + 32 * k), smem_desc(bh + 32 * k), idesc, true);
                umma_bf16(tmem, smem_desc(ah + 32 * k), smem_desc(bl + 32 * k), idesc, true);
            }
            umma_commit(empty + s);
        }
        if (ok) umma_commit(done);
    } else if (warp == 0 && lane == 0) {
        // ---------------- TMA producer
        int issued = 0;
        for (int kb = 0; kb < KB_LOAD; ++kb) {
            const int s = kb % STAGES;
            if (kb >= STAGES && !mbar_wait(empty + s, ((kb / STAGES) - 1) & 1, abort_flag)) {
                *abort_flag = 1;
                break;
            }
            uint8_t *a_dst = smem + s * STAGE_BYTES;
            uint8_t *b_dst = a_dst + A_STAGE_BYTES;
            const int pass = kb / KB1, kk = kb - pass * KB1;
            mbar_expect_tx(full + s, STAGE_BYTES);
            tma_load_2d(a_dst, &tmA, full + s, (pass == 1 ? K : 0) + kk * BK, m0);
            tma_load_2d(b_dst, &tmB, full + s, (pass == 2 ? K : 0) + kk * BK, n0);
            ++issued;
        }
        if (*abort_flag) {
            // let the copies already issued land before the CTA exits (bounded)
            for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb) {
                volatile int never = 0;
                mbar_wait(full + (kb % STAGES), (kb / STAGES) & 1, &never);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        const uint32_t idesc = f16 ? instr_desc_f16(BN) : instr_desc(BN);
        bool ok = true;
        for (int kb = 0; kb < KB; ++kb) {
            const int s = kb % STAGES;
            if (!mbar_wait(full + s, (kb / STAGES) & 1, abort_flag)) {
                *abort_flag = 1;
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t a_base = su32(smem + s * STAGE_BYTES);
            const uint32_t b_base = a_base + A_STAGE_BYTES;
#pragma unroll
            for (int k = 0; k < BK / 16; ++k)
                umma_bf16(tmem, smem_desc(a_base + 32 * k), smem_desc(b_base + 32 * k), idesc, (kb | k) != 0);
            umma_commit(empty + s);
        }
        if (ok) umma_commit(done);
    }
    __syncwarp();

    // ---------------- structure energies (B1, first N tile of each row block): warps 4..7,
    // idle during the main loop, one row per thread (gm_fixed.cuh); the block holds a ticket
    // and the last of the gridDim.y blocks writes energy[]
    if (EPI == EPI_B1 && e.energy != nullptr && blockIdx.x == 0 && warp >= 4) {
        const int m = m0 + (warp - 4) * 32 + lane;
        long long v[1] = {0};
        int b = -1;
        bool bad = false;
        if (m < e.n_atoms) {
            v[0] = to_fixed(atom_energy(m, e.species, e.n_species, e.sigma, e.mu, e.b3, e.nn_part, N / 32), bad);
            b = structure_of(e.atom_ptr, e.n_structures, m);
        }
        __shared__ int energy_last;
        warp_add_fixed<1>(b, v, 1, bad, e.red_acc, lane);
        __threadfence();
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (warp == 4 && lane == 0) {
            const unsigned long long ticket = atomicAdd(e.red_acc + (size_t)e.n_structures * RW, 1ull);
            energy_last = ticket == (unsigned long long)(gridDim.y - 1) ? 1 : 0;
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (energy_last)
            finalize_fixed(e.n_structures, 1, e.red_acc, e.energy, nullptr, threadIdx.x - 128, 128,
                           [] { asm volatile("bar.sync 1, 128;" ::: "memory"); });
    }

    // ---------------- epilogue: 8 warps; warp w reads TMEM lanes 32 (w % 4) .. +31 (rows)
    // and column half w / 4; thread = row m0 + 32 (w % 4) + lane
    const bool ready = __all_sync(0xffffffffu, mbar_wait(done, 0, abort_flag));
    tc_fence_after();
    if (ready) {
        // every MMA has completed, so the stage ring is free for the epilogue's staging
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const int quad = warp & 3, half = warp >> 2;
        const int row0 = m0 + quad * 32, m = row0 + lane;
        EpiStage &sg = *reinterpret_cast<EpiStage *>(smem + (size_t)warp * EPI_STAGE_BYTES);
        constexpr int CH = BN / 64;  // 32-column chunks per half
#pragma unroll 1
        for (int c = half * CH; c < (half + 1) * CH; ++c) {
            float v[32], part = 0.0f;
            tmem_ld_32cols(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(c * 32), v);
            epilogue32<EPI, ACT>(e, row0, n0 + c * 32, N, v, part, sg, lane);
            if (EPI == EPI_L2 || EPI == EPI_L2E) e.nn_part[(size_t)m * (N / 32) + (n0 + c * 32) / 32] = part;
        }
    } else if (threadIdx.x == 0) {
        set_status(status, GM_ERR_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

}  // namespace tc
}  // namespace gm
