// gm_mlp_fused.cuh -- the mixed path's four network GEMMs in one kernel per 128-row tile.
//
// For 128 atoms (rows) a CTA computes, with FP32 accumulators in TMEM,
//   L1  z1 = G W1          a1 = phi(z1 + b1) (BF16, kept in shared memory), phi' -> D1 (FP16)
//   L2  z2 = a1 W2         dZ2 = sigma_Z w3 phi'(z2 + b2) (FP16, in shared memory),
//                          partial sums of a2 . w3 per 32 columns -> nn_part (energies)
//   B1  dA1 = dZ2 W2^T     dZ1 = dA1 phi'(z1) (FP16, in shared memory)
//   B0  dG = dZ1 W1^T      -> dG (FP32), the input of the backward contraction
// (Eq. scale_shift and its gradient).  The activations of a layer never leave the SM: the
// shared-memory region X holds the current layer's A operand in the UMMA K-major 128-byte
// swizzled layout (written by the epilogue threads as TMA would have), and TMEM holds the
// accumulator.  The weights stream through a ring of shared-memory stages.
//
// Warps 0..7: epilogues (warp w reads TMEM lanes 32 (w % 4) .. +31, i.e. those rows, and
// column half w / 4).  Warp 8 lane 0: TMA producer (the G tile into X, then every weight tile
// of the four layers in order).  Warp 9 lane 0: MMA issuer.  Hand-offs are mbarriers: ring
// full/empty, g_full (the G tile landed), acc_full (a layer's MMAs completed; tcgen05.commit),
// x_ready (an epilogue wrote X and drained TMEM; 256 arrivals).  Every wait is bounded (one
// second, then GM_ERR_TIMEOUT); the MMA issuer waits for its own MMAs before the CTA frees TMEM.
#pragma once

#include "gm_gemm_tc.cuh"

namespace gm {
namespace tc {

struct FusedArgs {
    int M;                    // rows, a multiple of 128
    int n_atoms, n_species;
    const int32_t *species;
    const float *b1, *b2, *w3, *sigma;
    __half *D1;               // [M][H] phi'(z1) in FP16, written by L1's epilogue, read by B1's (same
                              // thread; it feeds an FP16 operand, dZ1 = dA1 phi'(z1), anyway), in a
                              // layout private to this kernel: per tile, 8-column groups g major,
                              // rows minor (d1_group), so a warp's 16-byte accesses are contiguous
    float *nn_part;           // [M][H/32]
    float *dG;                // [M][384] dE/dG, in the layout stage_rows reads as "tiled": per 128-row
                              // tile, 4-column groups major and rows minor
    int debug_stall;          // failure-reporting tests: the producer issues no loads at all
};

template <int H>
struct FusedShape {
    static constexpr int CHUNK = H >= 256 ? 256 : H;        // UMMA N of L1, L2, B1
    static constexpr int NCH = H / CHUNK;
    static constexpr int KBG = NFP / BK;                    // K blocks of L1 (384 / 64)
    static constexpr int KBH = H / BK;                      // K blocks of L2, B1, B0
    static constexpr int B0N = 128, B0CH = NFP / B0N;       // UMMA N and chunks of B0
    static constexpr int X_BYTES = (H > NFP ? H : NFP) * BM * 2;
    static constexpr int STAGE_BYTES = CHUNK * BK * 2;      // >= the B0 tiles (128 rows)
    static constexpr int STAGES = (232448 - 2048 - X_BYTES) / STAGE_BYTES < 8
                                      ? (232448 - 2048 - X_BYTES) / STAGE_BYTES : 8;
    static constexpr int TILES = NCH * KBG + 2 * NCH * KBH + B0CH * KBH;   // weight tiles streamed
    static constexpr size_t SMEM = (size_t)X_BYTES + (size_t)STAGES * STAGE_BYTES + 1024 + 256;
};

// 8 BF16 or FP16 values (16 bytes) of row r at column k0 of the K-major swizzled operand X
// (64-column blocks of 128 rows x 128 bytes; the 16-byte chunk j of row r sits at j ^ (r & 7))
__device__ __forceinline__ void x_store8(uint8_t *X, int r, int k0, uint4 v) {
    const int kb = k0 >> 6, j = (k0 & 63) >> 3;
    *reinterpret_cast<uint4 *>(X + (size_t)kb * (BM * 128) + r * 128 + ((j ^ (r & 7)) << 4)) = v;
}

// the 8 phi'(z1) values of row r (of the tile at m0) and column group g = column / 8
__device__ __forceinline__ uint4 *d1_group(__half *D1, int m0, int H, int g, int r) {
    return reinterpret_cast<uint4 *>(D1 + (size_t)m0 * H + ((size_t)g * BM + r) * 8);
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}

template <int H, int ACT>
__global__ void __launch_bounds__(320, 1)
    k_mlp_fused(const __grid_constant__ CUtensorMap tmG, const __grid_constant__ CUtensorMap tmW1,
                const __grid_constant__ CUtensorMap tmW2t, const __grid_constant__ CUtensorMap tmW2,
                const __grid_constant__ CUtensorMap tmW1p, FusedArgs f, int32_t *status) {
    using Sh = FusedShape<H>;
    constexpr int STAGES = Sh::STAGES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *X = smem;
    uint8_t *ring = smem + Sh::X_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(ring + (size_t)STAGES * Sh::STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *g_full = empty + STAGES;
    uint64_t *acc_full = g_full + 1;
    uint64_t *x_ready = acc_full + 1;
    uint64_t *drain = x_ready + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(g_full, 1);
        mbar_init(acc_full, 1);
        mbar_init(x_ready, 256);
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 8) {
        if (lane == 0) {
            // ---------------- TMA producer: the weights are parameters of the model (written
            // long before this launch), so their first stages are requested before the wait for
            // the preceding kernel; the G tile after it
            int issued = 0;
            auto tile = [&](int t) {
                const int s = t % STAGES;
                if (t >= STAGES && !mbar_wait(empty + s, ((t / STAGES) - 1) & 1, abort_flag)) return false;
                uint8_t *dst = ring + (size_t)s * Sh::STAGE_BYTES;
                int q = t;
                if (q < Sh::NCH * Sh::KBG) {                       // L1: W1 rows of chunk, K block
                    mbar_expect_tx(full + s, Sh::CHUNK * 128);
                    tma_load_2d(dst, &tmW1, full + s, (q % Sh::KBG) * BK, (q / Sh::KBG) * Sh::CHUNK);
                    return true;
                }
                q -= Sh::NCH * Sh::KBG;
                if (q < 2 * Sh::NCH * Sh::KBH) {                   // L2 (W2^T) then B1 (W2)
                    const CUtensorMap *mp = q < Sh::NCH * Sh::KBH ? &tmW2t : &tmW2;
                    q %= Sh::NCH * Sh::KBH;
                    mbar_expect_tx(full + s, Sh::CHUNK * 128);
                    tma_load_2d(dst, mp, full + s, (q % Sh::KBH) * BK, (q / Sh::KBH) * Sh::CHUNK);
                    return true;
                }
                q -= 2 * Sh::NCH * Sh::KBH;                        // B0 (W1^T), 128-row tiles
                mbar_expect_tx(full + s, Sh::B0N * 128);
                tma_load_2d(dst, &tmW1p, full + s, (q % Sh::KBH) * BK, (q / Sh::KBH) * Sh::B0N);
                return true;
            };
            if (!f.debug_stall) {
                for (; issued < STAGES && issued < Sh::TILES; ++issued) tile(issued);
                griddep_wait();
                mbar_expect_tx(g_full, Sh::KBG * BM * 128);
                for (int kb = 0; kb < Sh::KBG; ++kb) tma_load_2d(X + (size_t)kb * BM * 128, &tmG, g_full, kb * BK, m0);
                for (; issued < Sh::TILES; ++issued)
                    if (!tile(issued)) {
                        *abort_flag = 1;
                        break;
                    }
                if (*abort_flag) {
                    // let the copies already issued land before the CTA exits (bounded)
                    volatile int never = 0;
                    mbar_wait(g_full, 0, &never);
                    for (int t = (issued > STAGES ? issued - STAGES : 0); t < issued; ++t)
                        mbar_wait(full + (t % STAGES), (t / STAGES) & 1, &never);
                }
            }
        }
    } else if (warp == 9) {
        if (lane == 0) {
            // ---------------- MMA issuer
            bool ok = mbar_wait(g_full, 0, abort_flag);
            int t = 0;
            auto layer = [&](int nch, int kbs, int n, uint32_t idesc, int t_end) {
                for (int ch = 0; ch < nch && ok; ++ch)
                    for (int kb = 0; kb < kbs; ++kb) {
                        const int s = t % STAGES;
                        if (!mbar_wait(full + s, (t / STAGES) & 1, abort_flag)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a_base = su32(X + (size_t)kb * BM * 128);
                        const uint32_t b_base = su32(ring + (size_t)s * Sh::STAGE_BYTES);
#pragma unroll
                        for (int k = 0; k < BK / 16; ++k)
                            umma_bf16(tmem + (uint32_t)(ch * n), smem_desc(a_base + 32 * k), smem_desc(b_base + 32 * k),
                                      idesc, (kb | k) != 0);
                        umma_commit(empty + s);
                        ++t;
                    }
                (void)t_end;
                if (ok) umma_commit(acc_full);
            };
            auto wait_x = [&](int parity) {
                if (!ok) return;
                ok = mbar_wait(x_ready, parity, abort_flag);
                tc_fence_after();
            };
            if (ok) layer(Sh::NCH, Sh::KBG, Sh::CHUNK, instr_desc(Sh::CHUNK), 0);        // L1
            wait_x(0);
            if (ok) layer(Sh::NCH, Sh::KBH, Sh::CHUNK, instr_desc(Sh::CHUNK), 0);        // L2
            wait_x(1);
            if (ok) layer(Sh::NCH, Sh::KBH, Sh::CHUNK, instr_desc_f16(Sh::CHUNK), 0);    // B1
            wait_x(0);
            if (ok) layer(Sh::B0CH, Sh::KBH, Sh::B0N, instr_desc_f16(Sh::B0N), 0);       // B0
            if (!ok) *abort_flag = 1;
            // every MMA issued has completed before TMEM is freed
            umma_commit(drain);
            volatile int never = 0;
            mbar_wait(drain, 0, &never);
        }
    } else {
        // ---------------- epilogues: warps 0..7, thread = row m0 + 32 (warp % 4) + lane
        const int quad = warp & 3, half = warp >> 2;
        const int r = quad * 32 + lane, m = m0 + r;
        const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
        const int zi = m < f.n_atoms ? min(max(f.species[m], 0), f.n_species - 1) : 0;
        const float sg = m < f.n_atoms ? f.sigma[zi] : 0.0f;
        auto wait_acc = [&](int parity) {
            const bool ready = __all_sync(0xffffffffu, mbar_wait(acc_full, parity, abort_flag));
            tc_fence_after();
            return ready;
        };
        auto release_x = [&]() {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_fence_before();
            mbar_arrive(x_ready);
        };
        constexpr int CH32 = H / 64;          // 32-column chunks per column half
        bool ok = wait_acc(0);
        // the 32 biases (or output weights) of a column chunk: every lane of the warp reads the
        // same addresses, as eight 16-byte broadcast loads
        auto load32 = [](const float *p, float (&o)[32]) {
            const float4 *p4 = reinterpret_cast<const float4 *>(p);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float4 t = __ldg(p4 + q);
                o[4 * q] = t.x; o[4 * q + 1] = t.y; o[4 * q + 2] = t.z; o[4 * q + 3] = t.w;
            }
        };
        if (ok) {                             // E1: a1 -> X (BF16), phi'(z1) -> D1 (FP16)
            for (int c = half * CH32; c < (half + 1) * CH32; ++c) {
                float bias[32], v[32];
                load32(f.b1 + c * 32, bias);
                tmem_ld_32cols(tl + (uint32_t)(c * 32), v);
                float a[32], d[32];
#pragma unroll
                for (int t = 0; t < 32; ++t) a[t] = act_fast<ACT>(v[t] + bias[t], d[t]);
#pragma unroll
                for (int q = 0; q < 4; ++q) x_store8(X, r, c * 32 + 8 * q, pack8_bf16(a + 8 * q));
#pragma unroll
                for (int q = 0; q < 4; ++q) *d1_group(f.D1, m0, H, 4 * c + q, r) = pack8_f16(d + 8 * q);
            }
        }
        release_x();
        ok = ok && wait_acc(1);
        if (ok) {                             // E2: dZ2 -> X (FP16), energy partials
            for (int c = half * CH32; c < (half + 1) * CH32; ++c) {
                float bias[32], w3[32], v[32], y[32], part = 0.0f;
                load32(f.b2 + c * 32, bias);
                load32(f.w3 + c * 32, w3);
                tmem_ld_32cols(tl + (uint32_t)(c * 32), v);
#pragma unroll
                for (int t = 0; t < 32; ++t) {
                    float d;
                    const float a = act_fast<ACT>(v[t] + bias[t], d);
                    part = fmaf(a, w3[t], part);
                    y[t] = sg * w3[t] * d;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) x_store8(X, r, c * 32 + 8 * q, pack8_f16(y + 8 * q));
                f.nn_part[(size_t)m * (H / 32) + c] = part;
            }
        }
        release_x();
        ok = ok && wait_acc(0);
        if (ok) {                             // E3: dZ1 = dA1 phi'(z1) -> X (FP16)
            for (int c = half * CH32; c < (half + 1) * CH32; ++c) {
                float v[32], y[32];
                // this thread's phi'(z1) (written by itself in E1), loaded before the TMEM read
                // so that the two latencies overlap
                uint4 dq[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) dq[q] = *d1_group(f.D1, m0, H, 4 * c + q, r);
                tmem_ld_32cols(tl + (uint32_t)(c * 32), v);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const __half2 *h2 = reinterpret_cast<const __half2 *>(&dq[q]);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float2 d = __half22float2(h2[u]);
                        y[8 * q + 2 * u] = v[8 * q + 2 * u] * d.x;
                        y[8 * q + 2 * u + 1] = v[8 * q + 2 * u + 1] * d.y;
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) x_store8(X, r, c * 32 + 8 * q, pack8_f16(y + 8 * q));
            }
        }
        release_x();
        ok = ok && wait_acc(1);
        if (ok) {                             // E4: dG (FP32) -> global
            for (int c = half * 6; c < (half + 1) * 6; ++c) {
                float v[32];
                tmem_ld_32cols(tl + (uint32_t)(c * 32), v);
                float4 *dst = reinterpret_cast<float4 *>(f.dG + (size_t)m0 * NFP) + (size_t)(8 * c) * BM + r;
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    dst[(size_t)q * BM] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
        } else if (threadIdx.x == 0) {
            set_status(status, GM_ERR_TIMEOUT);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

}  // namespace tc
}  // namespace gm
