// gm_mlp_cluster.cuh -- the mixed path's four network GEMMs in one kernel, each 128-row tile
// split over a cluster of CS CTAs along the hidden width.
//
// Small systems have few 128-atom tiles (1536 atoms: 12), too few for one CTA per tile to
// fill the GPU.  Here CTA c of a tile's cluster owns hidden columns [c W, (c + 1) W) with
// W = H / CS and dG columns [c WG, (c + 1) WG) with WG = 384 / CS, and computes
//   L1  z1[:, slice] = G W1[:, slice]        a1 = phi(z1 + b1) (BF16), phi'(z1) -> D1 (FP16)
//   L2  z2[:, slice] = a1 W2[:, slice]       dZ2 = sigma_Z w3 phi'(z2 + b2) (FP16),
//                                           partial sums of a2 . w3 per 32 columns -> nn_part
//   B1  dA1[:, slice] = dZ2 W2[slice, :]^T   dZ1 = dA1 phi'(z1) (FP16)
//   B0  dG[:, gslice] = dZ1 W1[gslice, :]^T  -> dG (FP32)
// (Eq. scale_shift and its gradient).  L2, B1 and B0 contract over the whole hidden width, so
// after each of L1, L2 and B1 the cluster all-gathers the slices through L2: every CTA writes
// its slice (whole 64-column blocks of the UMMA K-major 128-byte-swizzled layout) into its own
// shared-memory region X, stores it with TMA to a global scratch array (L2-resident) and loads
// it back with one multicast TMA load into the same place of every other CTA's X.  (Copies from
// shared memory to shared memory across the cluster moved about 25 GB/s into each SM on B300,
// the multicast about 48 GB/s.)  The weights stream through a
// ring of stages (TMA), the accumulators live in TMEM.
//
// Ordering (all waits bounded: one second, then GM_ERR_TIMEOUT):
//   acc_full        the CTA's MMAs of a layer completed (tcgen05.commit)
//   x_free[g]       CS arrivals, one from every CTA of the cluster once its MMAs of layer g
//                   completed, so that gather g may overwrite every X (one barrier per gather)
//   x_full[d]       slice d of the current gather landed in X (the CTA's own slice: a local
//                   arrival; the others: the multicast load's complete_tx); the MMA issuer waits
//                   for each slice before its first K block, so MMAs on slices that have
//                   landed overlap the loads still in flight
// Before exit the cluster meets at a barrier, so that no CTA leaves while another may still
// arrive on its barriers or load into its shared memory; every CTA reaches it in bounded time
// because every wait before it is bounded.  The structure energies are then summed by the
// cluster's rank-0 CTA (fixed point, gm_fixed.cuh), whose barrier acquire makes the peers'
// partial sums visible.
//
// Warps 0..7: epilogues (warp w: TMEM lanes 32 (w % 4) .. +31 = those rows, column half w / 4;
// thread 0 also stores the slice and issues its multicast).  Warp 8 lane 0: TMA producer of the
// weights and the G tile.  Warp 9 lane 0: MMA issuer.
#pragma once

#include "gm_mlp_fused.cuh"

namespace gm {
namespace tc {

struct ClusterArgs {
    int M;                    // rows, a multiple of 128
    int n_atoms, n_species;
    const int32_t *species;
    const float *b1, *b2, *w3, *sigma;
    __half *D1;               // [M][H] phi'(z1) in FP16 (scratch)
    float *nn_part;           // [M][H/32]
    // the gathered layers go through [M][2H] scratch arrays (first H columns): a1, dZ2, dZ1
    float *dG;                // [M][384] dE/dG in the tiled layout of the per-tile kernel
    int debug_stall;          // failure-reporting tests: the producer issues no loads at all
    // structure energies (null energy: the caller sums them)
    const int32_t *atom_ptr;
    int n_structures;
    const float *mu, *b3;
    unsigned long long *red_acc;
    double *energy;
};

template <int H, int CS>
struct ClusterShape {
    static constexpr int W = H / CS;                        // hidden columns per CTA
    static constexpr int WG = NFP / CS;                     // dG columns per CTA
    static constexpr int KBG = NFP / BK, KBH = H / BK;
    static constexpr int KB_SLICE = W / BK;                 // K blocks of one CTA's slice
    static constexpr int NC = W / 64;                       // 32-column chunks per epilogue thread
    static constexpr bool KEEP_D = NC <= 2;                 // phi'(z1) stays in registers
    static constexpr int X_BYTES = (H > NFP ? H : NFP) * BM * 2;
    static constexpr int SLICE_BYTES = W * BM * 2;          // W / 64 whole K blocks of X
    static constexpr int ROWS = W > WG ? W : WG;
    static constexpr int STAGE_BYTES = ROWS * BK * 2;
    static constexpr int PARAM_BYTES = 3 * W * 4;           // the slice's b1, b2, w3
    static constexpr int AVAIL = 232448 - 2048 - X_BYTES - PARAM_BYTES;
    static constexpr int STAGES = AVAIL / STAGE_BYTES < 12 ? AVAIL / STAGE_BYTES : 12;
    static constexpr int TILES = KBG + 3 * KBH;
    static constexpr int TMEM_COLS = ROWS <= 64 ? 64 : (ROWS <= 128 ? 128 : 256);
    static constexpr size_t SMEM = (size_t)X_BYTES + (size_t)STAGES * STAGE_BYTES + PARAM_BYTES + 1024 + 1024;
    static_assert(W % 64 == 0 && W <= 256 && WG % 16 == 0 && WG <= 256, "cluster split");
    static_assert(STAGES >= 2, "stage ring");
};

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// shared::cluster address of the same variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cl_map(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ void cl_arrive(uint32_t remote_bar) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote_bar) : "memory");
}
// TMA store of one 64-column block of 128 rows from shared memory (same swizzled layout)
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, const void *src, int c_inner, int c_row) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(su32(src)), "r"(c_inner), "r"(c_row)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit_and_wait() {
    asm volatile("cp.async.bulk.commit_group;\n\tcp.async.bulk.wait_group 0;" ::: "memory");
}
// cluster barrier in two halves (every thread of every CTA arrives, then waits)
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire;" ::: "memory"); }
// TMA load of one box into the same shared-memory offset of every CTA in mask, each completing
// on its own barrier at the offset of bar
__device__ __forceinline__ void tma_load_2d_mc(void *dst, const CUtensorMap *map, uint64_t *bar, int c_inner,
                                               int c_row, uint16_t mask) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.multicast::cluster "
        "[%0], [%1, {%3, %4}], [%2], %5;" ::"r"(su32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(su32(bar)), "r"(c_inner), "r"(c_row), "h"(mask)
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cl(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait with cluster-scope acquire (the phase was completed by other CTAs' arrivals)
__device__ __forceinline__ bool mbar_wait_cl(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    if (mbar_try_wait_cl(bar, parity)) return true;
    const uint64_t t0 = now_ns();
    while (true) {
        if (mbar_try_wait_cl(bar, parity)) return true;
        if (*abort_flag) return false;
        if (now_ns() - t0 > WAIT_NS) return false;
    }
}
// 32 TMEM lanes x 16 consecutive 32-bit columns
__device__ __forceinline__ void tmem_ld_16cols(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

template <int H, int CS, int ACT>
__global__ void __launch_bounds__(320, 1)
    k_mlp_cluster(const __grid_constant__ CUtensorMap tmG, const __grid_constant__ CUtensorMap tmW1,
                  const __grid_constant__ CUtensorMap tmW2t, const __grid_constant__ CUtensorMap tmW2,
                  const __grid_constant__ CUtensorMap tmW1p, const __grid_constant__ CUtensorMap tmA1,
                  const __grid_constant__ CUtensorMap tmZ2, const __grid_constant__ CUtensorMap tmZ1, ClusterArgs f,
                  int32_t *status) {
    using Sh = ClusterShape<H, CS>;
    constexpr int STAGES = Sh::STAGES, W = Sh::W, WG = Sh::WG, NC = Sh::NC;
    extern __shared__ uint8_t smem_raw[];
    // the dynamic shared memory starts at the same offset in every CTA of the cluster, so the
    // aligned regions (and the barriers) sit at the same addresses in all of them
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *X = smem;
    uint8_t *ring = smem + Sh::X_BYTES;
    float *sb1 = reinterpret_cast<float *>(ring + (size_t)STAGES * Sh::STAGE_BYTES);
    float *sb2 = sb1 + W, *sw3 = sb2 + W;
    uint64_t *full = reinterpret_cast<uint64_t *>(sw3 + W);
    uint64_t *empty = full + STAGES;
    uint64_t *g_full = empty + STAGES;           // [KBG] one per K block of the G tile
    uint64_t *acc_full = g_full + Sh::KBG;
    uint64_t *x_full = acc_full + 1;             // [CS] one per source CTA's slice
    uint64_t *x_free = x_full + CS;              // [3] per gather
    uint64_t *drain = x_free + 3;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t cr = cluster_rank();
    const int m0 = (blockIdx.x / CS) * BM;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        for (int kb = 0; kb < Sh::KBG; ++kb) mbar_init(g_full + kb, 1);
        mbar_init(acc_full, 1);
        for (int d = 0; d < CS; ++d) mbar_init(x_full + d, 1);
        for (int g = 0; g < 3; ++g) mbar_init(x_free + g, CS);
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        tmem_alloc(tmem_slot, Sh::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    // every CTA's barriers are initialised before any CTA of the cluster signals or loads into
    // another: all threads arrive here and wait before their first such access (the producer
    // and MMA threads, which make none, only before the final barrier)
    cluster_arrive();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 8) {
        if (lane == 0) {
            // ---------------- TMA producer: this CTA's weight slices of the four layers in order
            // (first stages before the wait for the preceding kernel), the G tile after it
            int issued = 0;
            auto tile = [&](int t) {
                const int s = t % STAGES;
                if (t >= STAGES && !mbar_wait(empty + s, ((t / STAGES) - 1) & 1, abort_flag)) return false;
                uint8_t *dst = ring + (size_t)s * Sh::STAGE_BYTES;
                int q = t;
                if (q < Sh::KBG) {                                  // L1: W1^T rows of the slice
                    mbar_expect_tx(full + s, W * 128);
                    tma_load_2d(dst, &tmW1, full + s, q * BK, (int)cr * W);
                    return true;
                }
                q -= Sh::KBG;
                if (q < 2 * Sh::KBH) {                              // L2 (W2^T), then B1 (W2)
                    const CUtensorMap *mp = q < Sh::KBH ? &tmW2t : &tmW2;
                    mbar_expect_tx(full + s, W * 128);
                    tma_load_2d(dst, mp, full + s, (q % Sh::KBH) * BK, (int)cr * W);
                    return true;
                }
                q -= 2 * Sh::KBH;                                   // B0 (W1 rows of the dG slice)
                mbar_expect_tx(full + s, WG * 128);
                tma_load_2d(dst, &tmW1p, full + s, q * BK, (int)cr * WG);
                return true;
            };
            if (!f.debug_stall) {
                for (; issued < STAGES && issued < Sh::TILES; ++issued) tile(issued);
                griddep_wait();
                for (int kb = 0; kb < Sh::KBG; ++kb) {
                    mbar_expect_tx(g_full + kb, BM * 128);
                    tma_load_2d(X + (size_t)kb * BM * 128, &tmG, g_full + kb, kb * BK, m0);
                }
                for (; issued < Sh::TILES; ++issued)
                    if (!tile(issued)) {
                        *abort_flag = 1;
                        break;
                    }
                if (*abort_flag) {
                    // let the copies already issued land before the CTA exits (bounded)
                    volatile int never = 0;
                    for (int kb = 0; kb < Sh::KBG; ++kb) mbar_wait(g_full + kb, 0, &never);
                    for (int t = (issued > STAGES ? issued - STAGES : 0); t < issued; ++t)
                        mbar_wait(full + (t % STAGES), (t / STAGES) & 1, &never);
                }
            }
        }
        cluster_wait();
    } else if (warp == 9) {
        if (lane == 0) {
            // ---------------- MMA issuer.  The K blocks of a layer are issued in their natural
            // order; before the first K block of a slice the issuer waits for that slice (the
            // G tile block, or the source CTA's copy), so MMAs on slices that have landed
            // overlap the copies still in flight.
            bool ok = true;
            int t = 0;
            auto layer = [&](int kbs, uint32_t idesc, int xpar) {
                for (int kb = 0; kb < kbs && ok; ++kb) {
                    if (xpar < 0) {
                        ok = mbar_wait(g_full + kb, 0, abort_flag);
                    } else if (kb % Sh::KB_SLICE == 0) {
                        ok = mbar_wait_cl(x_full + kb / Sh::KB_SLICE, (uint32_t)xpar, abort_flag);
                    }
                    const int s = t % STAGES;
                    if (!ok || !mbar_wait(full + s, (t / STAGES) & 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a_base = su32(X + (size_t)kb * BM * 128);
                    const uint32_t b_base = su32(ring + (size_t)s * Sh::STAGE_BYTES);
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k)
                        umma_bf16(tmem, smem_desc(a_base + 32 * k), smem_desc(b_base + 32 * k), idesc, (kb | k) != 0);
                    umma_commit(empty + s);
                    ++t;
                }
                if (ok) umma_commit(acc_full);
            };
            layer(Sh::KBG, instr_desc(W), -1);          // L1 on the G tile
            layer(Sh::KBH, instr_desc(W), 0);           // L2 on a1
            layer(Sh::KBH, instr_desc_f16(W), 1);       // B1 on dZ2
            layer(Sh::KBH, instr_desc_f16(WG), 0);      // B0 on dZ1
            if (!ok) *abort_flag = 1;
            // every MMA issued has completed before TMEM is freed
            umma_commit(drain);
            volatile int never = 0;
            mbar_wait(drain, 0, &never);
        }
        cluster_wait();
    } else {
        // ---------------- epilogues: warps 0..7, thread = row m0 + 32 (warp % 4) + lane
        const int quad = warp & 3, half = warp >> 2;
        const int r = quad * 32 + lane, m = m0 + r;
        const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
        const int zi = m < f.n_atoms ? min(max(f.species[m], 0), f.n_species - 1) : 0;
        const float sg = m < f.n_atoms ? f.sigma[zi] : 0.0f;
        const int c0 = half * NC;                   // first chunk of this thread in the slice
        const int col0 = (int)cr * W;               // first hidden column of the slice
        // the slice's biases and output weights (model parameters), read from shared memory
        if (threadIdx.x < W) {
            sb1[threadIdx.x] = __ldg(f.b1 + col0 + threadIdx.x);
            sb2[threadIdx.x] = __ldg(f.b2 + col0 + threadIdx.x);
            sw3[threadIdx.x] = __ldg(f.w3 + col0 + threadIdx.x);
        }
        asm volatile("bar.sync 1, 256;" ::: "memory");
        cluster_wait();
        bool ok = true;
        // a failed wait stops the whole CTA (the abort word ends every other wait promptly)
        auto fail_if = [&](bool good) {
            if (!good) {
                ok = false;
                *abort_flag = 1;
            }
        };
        auto wait_acc = [&](int parity) {
            if (ok) fail_if(__all_sync(0xffffffffu, mbar_wait(acc_full, parity, abort_flag)));
            tc_fence_after();
        };
        // this CTA's MMAs of layer g have completed, so gather g may overwrite its X: tell every
        // CTA of the cluster (lane d of warp 0 tells CTA d; the arrivals travel in parallel)
        auto signal_free = [&](int g) {
            if (warp == 0 && lane < CS && ok) cl_arrive(cl_map(su32(x_free + g), (uint32_t)lane));
        };
        // the slice values of gather g are in registers: write the slice into X (this CTA's
        // MMAs may start on it); thread 0 stores it to the gather's global array and, once every
        // X of the cluster is free, multicasts it into the other CTAs' X
        auto publish = [&](int g, const CUtensorMap *map, const uint4 (&v)[NC][4]) {
            if (ok) {
#pragma unroll
                for (int c = 0; c < NC; ++c)
#pragma unroll
                    for (int q = 0; q < 4; ++q) x_store8(X, r, col0 + (c0 + c) * 32 + 8 * q, v[c][q]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("bar.sync 1, 256;" ::: "memory");
            if (threadIdx.x == 0 && ok && !*abort_flag) {
#pragma unroll 1
                for (int d = 0; d < CS; ++d) {
                    if (d == (int)cr) mbar_arrive(x_full + d);
                    else mbar_expect_tx(x_full + d, Sh::SLICE_BYTES);
                }
#pragma unroll 1
                for (int j = 0; j < Sh::KB_SLICE; ++j) {
                    const int kb = (int)cr * Sh::KB_SLICE + j;
                    tma_store_2d(map, X + (size_t)kb * BM * 128, kb * BK, m0);
                }
                bulk_commit_and_wait();          // the slice is in global memory
                if (mbar_wait_cl(x_free + g, 0, abort_flag)) {
                    const uint16_t others = (uint16_t)(((1u << CS) - 1u) & ~(1u << cr));
#pragma unroll 1
                    for (int j = 0; j < Sh::KB_SLICE; ++j) {
                        const int kb = (int)cr * Sh::KB_SLICE + j;
                        tma_load_2d_mc(X + (size_t)kb * BM * 128, map, x_full + cr, kb * BK, m0, others);
                    }
                } else {
                    *abort_flag = 1;
                }
            }
        };
        uint4 pk[NC][4];
        uint4 dk[Sh::KEEP_D ? NC : 1][4];           // phi'(z1) in FP16 when it stays in registers

        wait_acc(0);
        signal_free(0);
        if (ok) {                             // E1: a1 (BF16) -> X, phi'(z1) (FP16)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int lc = (c0 + c) * 32;
                float v[32], a[32], d[32];
                tmem_ld_32cols(tl + (uint32_t)lc, v);
#pragma unroll
                for (int u = 0; u < 32; ++u) a[u] = act_fast<ACT>(v[u] + sb1[lc + u], d[u]);
#pragma unroll
                for (int q = 0; q < 4; ++q) pk[c][q] = pack8_bf16(a + 8 * q);
                if constexpr (Sh::KEEP_D) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) dk[c][q] = pack8_f16(d + 8 * q);
                } else {
                    uint4 *dst = reinterpret_cast<uint4 *>(f.D1 + (size_t)m * H + col0 + lc);
#pragma unroll
                    for (int q = 0; q < 4; ++q) dst[q] = pack8_f16(d + 8 * q);
                }
            }
        }
        tc_fence_before();
        publish(0, &tmA1, pk);

        wait_acc(1);
        signal_free(1);
        if (ok) {                             // E2: dZ2 (FP16) -> X, energy partials
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int lc = (c0 + c) * 32;
                float v[32], y[32], part = 0.0f;
                tmem_ld_32cols(tl + (uint32_t)lc, v);
#pragma unroll
                for (int u = 0; u < 32; ++u) {
                    float d;
                    const float a = act_fast<ACT>(v[u] + sb2[lc + u], d);
                    part = fmaf(a, sw3[lc + u], part);
                    y[u] = sg * sw3[lc + u] * d;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) pk[c][q] = pack8_f16(y + 8 * q);
                f.nn_part[(size_t)m * (H / 32) + (col0 + lc) / 32] = part;
            }
        }
        tc_fence_before();
        publish(1, &tmZ2, pk);

        if constexpr (!Sh::KEEP_D) {
            // this thread's phi'(z1) (written by itself in E1), loaded before the TMEM read
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const uint4 *dsrc = reinterpret_cast<const uint4 *>(f.D1 + (size_t)m * H + col0 + (c0 + c) * 32);
#pragma unroll
                for (int q = 0; q < 4; ++q) pk[c][q] = dsrc[q];
            }
        }
        wait_acc(0);
        signal_free(2);
        if (ok) {                             // E3: dZ1 = dA1 phi'(z1) (FP16) -> X
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                float v[32], y[32];
                tmem_ld_32cols(tl + (uint32_t)((c0 + c) * 32), v);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint4 dq = Sh::KEEP_D ? dk[Sh::KEEP_D ? c : 0][q] : pk[c][q];
                    const __half2 *h2 = reinterpret_cast<const __half2 *>(&dq);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float2 d = __half22float2(h2[u]);
                        y[8 * q + 2 * u] = v[8 * q + 2 * u] * d.x;
                        y[8 * q + 2 * u + 1] = v[8 * q + 2 * u + 1] * d.y;
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) pk[c][q] = pack8_f16(y + 8 * q);
            }
        }
        tc_fence_before();
        publish(2, &tmZ1, pk);

        wait_acc(1);
        if (ok) {                             // E4: dG slice (FP32) -> global, 16-column chunks
            constexpr int N16 = WG / 16, H0 = (N16 + 1) / 2;
            const int q0 = half ? H0 : 0, q1 = half ? N16 : H0;
            for (int q = q0; q < q1; ++q) {
                float v[16];
                tmem_ld_16cols(tl + (uint32_t)(q * 16), v);
                // tiled layout (4-column groups major, rows minor per 128-row tile), as the
                // per-tile kernel writes it: a warp's stores are 512 contiguous bytes
                float4 *dst = reinterpret_cast<float4 *>(f.dG + (size_t)m0 * NFP) +
                              (size_t)((cr * WG + q * 16) / 4) * BM + (m - m0);
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    dst[(size_t)u * BM] = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
            }
        }
        if (!ok && threadIdx.x == 0) set_status(status, GM_ERR_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, Sh::TMEM_COLS);
    if (*abort_flag && threadIdx.x == 0) set_status(status, GM_ERR_TIMEOUT);
    // no CTA leaves while another may still arrive on its barriers or load into its shared
    // memory; the barrier's release/acquire also makes every CTA's nn_part visible to rank 0
    cluster_arrive();
    cluster_wait();
    if (status_bad(status)) {
        // a wait gave up somewhere: a multicast issued just before it may still be landing in
        // this CTA's shared memory (loads take microseconds; this CTA stays 50 us longer)
        const uint64_t t0 = now_ns();
        while (now_ns() - t0 < 50000ull) __nanosleep(1000);
    }

    // ---------------- structure energies: rank 0 of the cluster, warps 0..3, one row each
    if (f.energy != nullptr && cr == 0 && warp < 4) {
        const int m = m0 + warp * 32 + lane;
        long long v[1] = {0};
        int b = -1;
        bool bad = false;
        if (m < f.n_atoms && !status_bad(status)) {
            float2 pt[H / 64];
            const float2 *row = reinterpret_cast<const float2 *>(f.nn_part + (size_t)m * (H / 32));
#pragma unroll
            for (int t = 0; t < H / 64; ++t) pt[t] = __ldcg(row + t);
            float nn = f.b3[0];
#pragma unroll
            for (int t = 0; t < H / 64; ++t) {
                nn += pt[t].x;
                nn += pt[t].y;
            }
            const int z = min(max(f.species[m], 0), f.n_species - 1);
            v[0] = to_fixed(fmaf(f.sigma[z], nn, f.mu[z]), bad);
            b = structure_of(f.atom_ptr, f.n_structures, m);
        }
        __shared__ int energy_last;
        warp_add_fixed<1>(b, v, 1, bad, f.red_acc, lane);
        __threadfence();
        asm volatile("bar.sync 2, 128;" ::: "memory");
        if (threadIdx.x == 0) {
            const unsigned long long ticket = atomicAdd(f.red_acc + (size_t)f.n_structures * RW, 1ull);
            energy_last = ticket == (unsigned long long)(gridDim.x / CS - 1) ? 1 : 0;
        }
        asm volatile("bar.sync 2, 128;" ::: "memory");
        if (energy_last)
            finalize_fixed(f.n_structures, 1, f.red_acc, f.energy, nullptr, threadIdx.x, 128,
                           [] { asm volatile("bar.sync 2, 128;" ::: "memory"); });
    }
}

}  // namespace tc
}  // namespace gm
