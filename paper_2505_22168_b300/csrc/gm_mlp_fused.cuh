// gm_mlp_fused.cuh -- the mixed path's four network GEMMs in one persistent kernel over
// 128-row tiles.
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
// accumulator.  The weights stream through a ring of shared-memory stages.  One CTA per SM
// takes tiles blockIdx.x, blockIdx.x + gridDim.x, ...
//
// Warps 0..7: epilogues (warp w reads TMEM lanes 32 (w % 4) .. +31, i.e. those rows).  Warp 8
// lane 0: TMA producer (per tile its G into X and every weight tile of the four layers in
// order).  Warp 9 lane 0: MMA issuer.  The epilogue of a layer runs in two halves of its
// columns, and the tensor cores do not wait for a whole epilogue: the next layer's first K
// blocks (X columns of half 0) run while the epilogue does half 1, and the epilogue of a
// layer starts on half 0 (its own chunk of accumulator columns at H = 512) while the MMAs of
// half 1 still run, writing X once the layer's MMAs have read its first K blocks.  The next
// tile's G loads into X while the last epilogue (dG) runs.  Hand-offs are mbarriers: ring
// full/empty, g_full, x_free (B0 done with X), accb[layer][half] and xlo[layer]
// (tcgen05.commit), xh[layer][half] (an epilogue half wrote X and read its TMEM columns; 256
// arrivals).  Every barrier completes one phase per tile.  Every wait is bounded (one second,
// then GM_ERR_TIMEOUT); the MMA issuer waits for its own MMAs before the CTA frees TMEM.
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
    // B0 (N = 384) in chunks of 256 + 128 columns when a stage holds 256 weight rows, else 3 x 128
    static constexpr bool B0_WIDE = CHUNK >= 256;
    static constexpr int B0CH = B0_WIDE ? 2 : 3;
    static constexpr __host__ __device__ int b0_col(int ch) { return ch * (B0_WIDE ? 256 : 128); }
    static constexpr __host__ __device__ int b0_n(int ch) { return B0_WIDE && ch == 0 ? 256 : 128; }
    static constexpr int X_BYTES = (H > NFP ? H : NFP) * BM * 2;
    static constexpr int STAGE_BYTES = CHUNK * BK * 2;      // one weight tile (B0's too, asserted below)
    static constexpr int STAGES = (232448 - 2048 - X_BYTES) / STAGE_BYTES < 8
                                      ? (232448 - 2048 - X_BYTES) / STAGE_BYTES : 8;
    static constexpr int TILES = NCH * KBG + 2 * NCH * KBH + B0CH * KBH;   // weight tiles per row tile
    static_assert(STAGE_BYTES >= b0_n(0) * BK * 2, "a stage holds a B0 weight tile");
    static constexpr size_t SMEM = (size_t)X_BYTES + (size_t)STAGES * STAGE_BYTES + 1024 + 512;
    static constexpr int KH = H / 128;                      // X blocks written by one epilogue half
    static constexpr int HW = H / 4;                        // columns of one warp in an epilogue half
    // B0's first chunk overwrites TMEM columns that E3's second half reads (then both E3 halves
    // precede its first MMA)
    static constexpr bool B0_AFTER_E3 = b0_n(0) > H / 2;
    // TMEM column base of each layer's accumulator: at H = 512 every layer fills TMEM; narrower
    // networks put L2 at column 256 so that its MMAs need not wait for E1's second half
    static constexpr __host__ __device__ int base(int l) { return (H <= 256 && l == 1) ? 256 : 0; }
};
static_assert(FusedShape<512>::SMEM <= 232448 && FusedShape<256>::SMEM <= 232448 && FusedShape<128>::SMEM <= 232448,
              "fused network kernel fits in shared memory");
static_assert((2 * 8 + 22) * 8 + 8 <= 512, "barriers, TMEM slot and abort flag fit in the 512-byte tail");

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

// L2 prefetch of one box of a tiled tensor (no shared-memory destination, no barrier)
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap *map, int c_inner, int c_row) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(reinterpret_cast<uint64_t>(map)),
                 "r"(c_inner), "r"(c_row)
                 : "memory");
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
    constexpr int STAGES = Sh::STAGES, KH = Sh::KH, HW = Sh::HW;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *X = smem;
    uint8_t *ring = smem + Sh::X_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(ring + (size_t)STAGES * Sh::STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *g_full = empty + STAGES;      // the tile's G landed in X
    uint64_t *x_free = g_full + 1;          // B0 no longer reads X (MMA -> producer)
    uint64_t *accb = x_free + 1;            // [layer][half]: the half's accumulator columns are final
    uint64_t *xlo = accb + 8;               // [layer < 3]: the layer no longer reads X blocks [0, KH)
    uint64_t *xh = xlo + 3;                 // [layer][half]: that epilogue half is done (256 arrivals)
    uint64_t *drain = xh + 8;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = f.M / BM;
    const int my_tiles = (int)blockIdx.x < n_tiles ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(g_full, 1);
        mbar_init(x_free, 1);
        for (int i = 0; i < 8; ++i) mbar_init(accb + i, 1);
        for (int i = 0; i < 3; ++i) mbar_init(xlo + i, 1);
        for (int i = 0; i < 8; ++i) mbar_init(xh + i, 256);
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
        if (lane == 0 && !f.debug_stall) {
            // ---------------- TMA producer: per tile the first STAGES weight tiles (their
            // slots free up while the previous tile's B0 runs), then the tile's G into X once
            // B0 no longer reads it, then the rest of the weights.  The weights are parameters
            // of the model, so the first tile's first stages go out before the wait for the
            // preceding kernel.
            int issued = 0, g_issued = 0;
            bool ok = true;
            auto tile = [&](int j) {
                const int s = j % STAGES;
                if (j >= STAGES && !mbar_wait(empty + s, ((j / STAGES) - 1) & 1, abort_flag)) return false;
                uint8_t *dst = ring + (size_t)s * Sh::STAGE_BYTES;
                int q = j % Sh::TILES;
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
                q -= 2 * Sh::NCH * Sh::KBH;                        // B0 (W1^T) in 128-row boxes
                const int ch = q / Sh::KBH, kb = q % Sh::KBH;
                mbar_expect_tx(full + s, Sh::b0_n(ch) * 128);
                for (int r0 = 0; r0 < Sh::b0_n(ch); r0 += 128)
                    tma_load_2d(dst + (size_t)r0 * 128, &tmW1p, full + s, kb * BK, Sh::b0_col(ch) + r0);
                return true;
            };
            for (int it = 0; it < my_tiles && ok; ++it) {
                const int m0 = ((int)blockIdx.x + it * (int)gridDim.x) * BM;
                const int j0 = it * Sh::TILES;
                while (ok && issued < j0 + (STAGES < Sh::TILES ? STAGES : Sh::TILES)) {
                    if (!tile(issued)) ok = false;
                    else ++issued;
                }
                if (!ok) break;
                if (it == 0) griddep_wait();
                else if (!mbar_wait(x_free, (it - 1) & 1, abort_flag)) {
                    ok = false;
                    break;
                }
                mbar_expect_tx(g_full, Sh::KBG * BM * 128);
                for (int kb = 0; kb < Sh::KBG; ++kb) tma_load_2d(X + (size_t)kb * BM * 128, &tmG, g_full, kb * BK, m0);
                ++g_issued;
                if (it + 1 < my_tiles)                             // the next tile's G into L2
                    for (int kb = 0; kb < Sh::KBG; ++kb) tma_prefetch_2d(&tmG, kb * BK, m0 + (int)gridDim.x * BM);
                while (ok && issued < j0 + Sh::TILES) {
                    if (!tile(issued)) ok = false;
                    else ++issued;
                }
            }
            if (!ok) {
                *abort_flag = 1;
                // let the copies already issued land before the CTA exits (bounded)
                volatile int never = 0;
                if (g_issued > 0) mbar_wait(g_full, (g_issued - 1) & 1, &never);
                for (int t = (issued > STAGES ? issued - STAGES : 0); t < issued; ++t)
                    mbar_wait(full + (t % STAGES), (t / STAGES) & 1, &never);
            }
        }
    } else if (warp == 9) {
        if (lane == 0) {
            // ---------------- MMA issuer.  A layer's chunk c accumulates into TMEM columns
            // base + c n; before its first MMA the epilogue half that last read those columns
            // must be done, and K blocks [0, KH) / [KH, ..) of X need the previous epilogue's
            // half 0 / half 1.  Commits: accb after the chunk(s) holding each epilogue half,
            // xlo after the last chunk's K block KH - 1, x_free after B0.
            bool ok = true;
            int t = 0;
            auto kblock = [&](uint32_t d, int kb, uint32_t idesc) {
                const int s = t % STAGES;
                if (!mbar_wait(full + s, (t / STAGES) & 1, abort_flag)) return false;
                tc_fence_after();
                const uint32_t a_base = su32(X + (size_t)kb * BM * 128);
                const uint32_t b_base = su32(ring + (size_t)s * Sh::STAGE_BYTES);
#pragma unroll
                for (int k = 0; k < BK / 16; ++k)
                    umma_bf16(d, smem_desc(a_base + 32 * k), smem_desc(b_base + 32 * k), idesc, (kb | k) != 0);
                umma_commit(empty + s);
                ++t;
                return true;
            };
            auto wait_bar = [&](uint64_t *bar, uint32_t parity) {
                if (!ok) return;
                ok = mbar_wait(bar, parity, abort_flag);
                tc_fence_after();
            };
            for (int it = 0; it < my_tiles && ok; ++it) {
                const uint32_t par = it & 1;
                // L1 (X = G, KBG blocks)
                wait_bar(g_full, par);
                for (int ch = 0; ch < Sh::NCH && ok; ++ch) {
                    if (it > 0) wait_bar(xh + 6 + ch, par ^ 1);   // the previous tile's E4 half ch
                    for (int kb = 0; kb < Sh::KBG && ok; ++kb) {
                        ok = kblock(tmem + (uint32_t)(Sh::base(0) + ch * Sh::CHUNK), kb, instr_desc(Sh::CHUNK));
                        if (ok && ch == Sh::NCH - 1 && kb == KH - 1) umma_commit(xlo + 0);
                    }
                    if (ok && ch == 0) umma_commit(accb + 0);
                    if (ok && ch == Sh::NCH - 1) umma_commit(accb + 1);
                }
                // L2 (X = a1), B1 (X = dZ2, FP16)
                for (int l = 1; l <= 2 && ok; ++l) {
                    const uint32_t idesc = l == 1 ? instr_desc(Sh::CHUNK) : instr_desc_f16(Sh::CHUNK);
                    for (int ch = 0; ch < Sh::NCH && ok; ++ch) {
                        for (int kb = 0; kb < Sh::KBH && ok; ++kb) {
                            if (ch == 0 && kb == 0) wait_bar(xh + 2 * (l - 1), par);
                            if (ch == 0 && kb == KH) wait_bar(xh + 2 * (l - 1) + 1, par);
                            if (!ok) break;
                            ok = kblock(tmem + (uint32_t)(Sh::base(l) + ch * Sh::CHUNK), kb, idesc);
                            if (ok && ch == Sh::NCH - 1 && kb == KH - 1) umma_commit(xlo + l);
                        }
                        if (ok && ch == 0) umma_commit(accb + 2 * l);
                        if (ok && ch == Sh::NCH - 1) umma_commit(accb + 2 * l + 1);
                    }
                }
                // B0 (X = dZ1, FP16) at TMEM column 0: its chunks end at columns 256 and 384 (E4's
                // halves)
                for (int ch = 0; ch < Sh::B0CH && ok; ++ch) {
                    const uint32_t idesc = instr_desc_f16(Sh::b0_n(ch));
                    for (int kb = 0; kb < Sh::KBH && ok; ++kb) {
                        if (ch == 0 && kb == 0) {
                            wait_bar(xh + 4, par);
                            if (Sh::B0_AFTER_E3) wait_bar(xh + 5, par);
                        }
                        if (!Sh::B0_AFTER_E3 && ch == 0 && kb == KH) wait_bar(xh + 5, par);
                        if (!ok) break;
                        ok = kblock(tmem + (uint32_t)Sh::b0_col(ch), kb, idesc);
                    }
                    if (ok && Sh::b0_col(ch) + Sh::b0_n(ch) == 256) umma_commit(accb + 6);
                    if (ok && ch == Sh::B0CH - 1) {
                        umma_commit(accb + 7);
                        umma_commit(x_free);
                    }
                }
            }
            if (!ok) *abort_flag = 1;
            // every MMA issued has completed before TMEM is freed
            umma_commit(drain);
            volatile int never = 0;
            mbar_wait(drain, 0, &never);
        }
    } else {
        // ---------------- epilogues: warps 0..7, thread = tile row 32 (warp % 4) + lane.  Each
        // layer's epilogue runs in two halves of its columns (E4: [0, 256) and [256, 384)); warp
        // w takes the quarter w / 4 of each half, the same columns in E1 and E3 (phi'(z1) is
        // private to the thread).
        const int quad = warp & 3, wq = warp >> 2;
        const int r = quad * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
        bool ok = true;
        auto wait_acc = [&](uint64_t *bar, uint32_t parity) {
            if (ok) ok = __all_sync(0xffffffffu, mbar_wait(bar, parity, abort_flag));
            tc_fence_after();
        };
        auto release = [&](uint64_t *bar) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_fence_before();
            mbar_arrive(bar);
        };
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
        for (int it = 0; it < my_tiles && ok; ++it) {
            const uint32_t par = it & 1;
            const int m0 = ((int)blockIdx.x + it * (int)gridDim.x) * BM, m = m0 + r;
            const int zi = m < f.n_atoms ? min(max(f.species[m], 0), f.n_species - 1) : 0;
            const float sg = m < f.n_atoms ? f.sigma[zi] : 0.0f;
            for (int h = 0; h < 2 && ok; ++h) {      // E1: a1 -> X (BF16), phi'(z1) -> D1 (FP16)
                wait_acc(accb + h, par);
                if (h == 0) wait_acc(xlo + 0, par);
                if (!ok) break;
#pragma unroll 1
                for (int col = h * (H / 2) + wq * HW; col < h * (H / 2) + (wq + 1) * HW; col += 32) {
                    float bias[32], v[32];
                    load32(f.b1 + col, bias);
                    tmem_ld_32cols(tl + (uint32_t)(Sh::base(0) + col), v);
                    float a[32], d[32];
#pragma unroll
                    for (int u = 0; u < 32; ++u) a[u] = act_fast<ACT>(v[u] + bias[u], d[u]);
#pragma unroll
                    for (int q = 0; q < 4; ++q) x_store8(X, r, col + 8 * q, pack8_bf16(a + 8 * q));
#pragma unroll
                    for (int q = 0; q < 4; ++q) *d1_group(f.D1, m0, H, col / 8 + q, r) = pack8_f16(d + 8 * q);
                }
                release(xh + h);
            }
            for (int h = 0; h < 2 && ok; ++h) {      // E2: dZ2 -> X (FP16), energy partials
                wait_acc(accb + 2 + h, par);
                if (h == 0) wait_acc(xlo + 1, par);
                if (!ok) break;
#pragma unroll 1
                for (int col = h * (H / 2) + wq * HW; col < h * (H / 2) + (wq + 1) * HW; col += 32) {
                    float bias[32], w3[32], v[32], y[32], part = 0.0f;
                    load32(f.b2 + col, bias);
                    load32(f.w3 + col, w3);
                    tmem_ld_32cols(tl + (uint32_t)(Sh::base(1) + col), v);
#pragma unroll
                    for (int u = 0; u < 32; ++u) {
                        float d;
                        const float a = act_fast<ACT>(v[u] + bias[u], d);
                        part = fmaf(a, w3[u], part);
                        y[u] = sg * w3[u] * d;
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) x_store8(X, r, col + 8 * q, pack8_f16(y + 8 * q));
                    f.nn_part[(size_t)m * (H / 32) + col / 32] = part;
                }
                release(xh + 2 + h);
            }
            for (int h = 0; h < 2 && ok; ++h) {      // E3: dZ1 = dA1 phi'(z1) -> X (FP16)
                wait_acc(accb + 4 + h, par);
                if (h == 0) wait_acc(xlo + 2, par);
                if (!ok) break;
#pragma unroll 1
                for (int col = h * (H / 2) + wq * HW; col < h * (H / 2) + (wq + 1) * HW; col += 32) {
                    float v[32], y[32];
                    // this thread's phi'(z1) (written by itself in E1), loaded before the TMEM
                    // read so that the two latencies overlap
                    uint4 dq[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) dq[q] = *d1_group(f.D1, m0, H, col / 8 + q, r);
                    tmem_ld_32cols(tl + (uint32_t)(Sh::base(2) + col), v);
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
                    for (int q = 0; q < 4; ++q) x_store8(X, r, col + 8 * q, pack8_f16(y + 8 * q));
                }
                release(xh + 4 + h);
            }
            for (int h = 0; h < 2 && ok; ++h) {      // E4: dG (FP32) -> global, tiled
                wait_acc(accb + 6 + h, par);
                if (!ok) break;
                const int c0 = h == 0 ? wq * 128 : 256 + wq * 64, c1 = h == 0 ? c0 + 128 : c0 + 64;
#pragma unroll 1
                for (int col = c0; col < c1; col += 32) {
                    float v[32];
                    tmem_ld_32cols(tl + (uint32_t)col, v);
                    float4 *dst = reinterpret_cast<float4 *>(f.dG + (size_t)m0 * NFP) + (size_t)(col / 4) * BM + r;
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        dst[(size_t)q * BM] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
                release(xh + 6 + h);
            }
        }
        if (!ok) {
            *abort_flag = 1;
            if (lane == 0) set_status(status, GM_ERR_TIMEOUT);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

}  // namespace tc
}  // namespace gm
