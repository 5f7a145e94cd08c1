// gm_nlist.cu -- cell-list neighbour search for batches of periodic orthorhombic boxes.
//
// Neighbour rule (section "Deployment": the neighbour list covers every periodic image
// inside the cutoff, also when the cell is so small that an atom sees several images of
// the same neighbour): all (i, j, n) with |r'_j - r'_i + n L| < r_cut except (j == i,
// n == 0), where r' are positions wrapped into [0, L) per axis.  The membership decision
// is taken in FP64 with correctly rounded operations in a fixed order (bit-identical to
// the oracle); an FP32 distance filter decides every candidate that lies clearly inside
// or outside a band around r_cut^2 whose half-width bounds the FP32 rounding error, so
// FP64 arithmetic (slow on B300) runs only for the rare candidates inside the band.
//
// Phases (one stream, no host synchronisation):
//   setup    per-structure cell grid (cells >= r_cut, at most max(1, n_atoms) cells) and
//            the global cell numbering; zero the cell histograms
//   bin      wrap positions, cell index, atomic histogram
//   scan     cell offsets (block chunks, then the carry of the earlier chunks)
//   scatter  atoms into cells (atomic slots)
//   sort     one warp per cell packs the cell's FP32 wrapped positions in ascending atom
//            index (float4, index in w)
//   count    one warp per work item (a home cell, or one of `split` interleaved parts of its
//            atoms): the lanes take 32 candidates of the 27 stencil cells (each with its
//            periodic image) at a time and test them against every home atom of the item
//   scan     row offsets; n_pairs and the capacity check
//   fill     the count pass again, writing col and shift through a ballot prefix
// The row order is stencil cell (dz, dy, dx ascending) then ascending neighbour index, the
// same in both passes.  Structures whose box is shorter than r_cut along some axis (several
// images of a cell per stencil direction) take a per-atom loop over the stencil instead.
// Scans of up to NL_SCAN_ONE_BLOCK entries run in one block.
//
// All phases run in ONE cooperative launch with grid-wide barriers between them (each a
// bounded wait: after about one second it records GM_ERR_TIMEOUT and the kernel returns),
// or, selected by a tuning knob, as one launch per phase.
#include <math.h>

#include <optional>

#include "gm_internal.h"

namespace gm {

constexpr int NL_THREADS = 256;
constexpr int NL_WARPS = NL_THREADS / 32;
constexpr int NL_SCAN_SUB = NL_THREADS * 4;
constexpr int NL_SCAN_ONE_BLOCK = 4096;
constexpr int NL_HOME_STENCIL = 13;     // (0, 0, 0) in the 27-cell stencil
constexpr int NL_MAX_BLOCKS = 4096;

// Per-structure cell-list geometry (device, in the neighbour workspace).
struct NlStruct {
    double L[3];      // orthorhombic box edges
    double invL[3];   // 1 / L (rounded): wrap fast path
    double inv_cs[3]; // cells per unit length (cell edge >= r_cut unless the box is smaller)
    int nc[3];        // cells per axis
    int K[3];         // stencil half-width per axis (cells)
    int cell0;        // first global cell index of this structure
    int a0, n;        // atoms
    float Lf[3];      // edges in FP32 (distance filter)
    float eps2;       // half-width of the FP32 band around r_cut^2 decided in FP64
};

// Per-axis integers as three signed bytes (x | y << 8 | z << 16); bit 31 marks a value
// outside -127..127 (the consumer then works with the full integers).
constexpr unsigned NL_FAR = 0x80000000u;
__device__ __forceinline__ unsigned bytes3(int x, int y, int z) {
    const bool ok = x >= -127 && x <= 127 && y >= -127 && y <= 127 && z >= -127 && z <= 127;
    return ok ? ((unsigned)(x & 255) | ((unsigned)(y & 255) << 8) | ((unsigned)(z & 255) << 16)) : NL_FAR;
}
__device__ __forceinline__ int byte_at(unsigned p, int axis) { return (int)(signed char)((p >> (8 * axis)) & 255u); }

// Slab entries hold the shift as a code 0..26 of (s0, s1, s2) in {-1, 0, 1}^3; NL_NOCODE
// for any other shift (its row is searched again during the compaction).
constexpr unsigned NL_NOCODE = 31u;
__device__ __forceinline__ unsigned shift_code(unsigned sb) {
    if (sb & NL_FAR) return NL_NOCODE;
    const int s0 = byte_at(sb, 0), s1 = byte_at(sb, 1), s2 = byte_at(sb, 2);
    const bool ok = s0 >= -1 && s0 <= 1 && s1 >= -1 && s1 <= 1 && s2 >= -1 && s2 <= 1;
    return ok ? (unsigned)((s0 + 1) + 3 * (s1 + 1) + 9 * (s2 + 1)) : NL_NOCODE;
}

// a + b per byte for two bytes3 values; NL_FAR if either is far or a sum leaves -127..127
__device__ __forceinline__ unsigned bytes3_add(unsigned a, unsigned b) {
    if ((a | b) & NL_FAR) return NL_FAR;
    const unsigned s = __vadd4(a, b);
    const bool wrapped = __vaddss4(a, b) != s;
    const bool minus128 = __vcmpeq4(s | 0xFF000000u, 0x80808080u) != 0u;
    return (wrapped || minus128) ? NL_FAR : s;
}

struct NlArgs {
    int N, B, n_species, ncmax, split;
    const int32_t *atom_ptr;
    const double *pos;
    const int32_t *species;
    const double *cell;
    const uint8_t *pbc;
    double rc;
    float rc2f;
    NlStruct *S;
    int32_t *ncells;        // device scalar: cells of all structures
    int32_t *cellid, *ccount, *cstart, *cfill, *unsorted, *counts, *bsum, *mimg;
    int32_t *cstruct;       // structure of each cell (filled while binning)
    int32_t *item_ctr;      // [2] work-item counters of the block-level search passes (zeroed per build)
    uint32_t *xsm;          // image counts of the sorted atoms (bytes3 of mimg)
    uint32_t *mpk;          // image counts by atom index (bytes3 of mimg)
    uint32_t *slab;         // single-pass search: row i at i * maxn, entries j | shift code << 27
    int maxn;               // slab row length (0: two-pass search, no slab)
    int block_items;        // 1: block-level search items, 0: warp-level
    int small;              // cooperative launch: grids and short scans computed by every block
    int mid;                // cooperative launch, N + B up to 8192 (not small): the brute-force search
                            // if the boxes allow it, else the phases of large systems
    int try_brute;          // small systems: brute-force search when every box is single-image
    int *brute_over;        // set when a brute-force row exceeds BR_CAP (zeroed per build)
    uint8_t *redo;          // 1: row searched again during the compaction
    int32_t *redo_list, *n_redo;
    double *xw;
    float4 *xs;
    int32_t *row_ptr, *col;
    char4 *shift;
    int64_t cap;
    int64_t *n_pairs;
    unsigned *bar;          // grid barrier: [0] arrivals, [1] generation
    int32_t *status;
    const int32_t *gate;    // if not null: build only when *gate != 0 (written by an earlier kernel)
    int debug_stall;        // tests of failure reporting: block 0 returns before the first barrier
};

// A gated build (the skin test of an MD step decides on the device whether the list is
// rebuilt): every block reads the same word and returns before its first barrier.
__device__ __forceinline__ bool nl_gated_off(const NlArgs &a) {
    return a.gate != nullptr && *reinterpret_cast<const volatile int32_t *>(a.gate) == 0;
}

__device__ __forceinline__ unsigned long long nl_clock_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of a cooperative launch (all blocks co-resident).  Thread 0 of each block
// reads the generation, arrives with a release-acquire increment (the block's writes were
// ordered before it by the block barrier), and waits with acquire loads until the last
// arrival resets the count and advances the generation.  The wait is bounded: on expiry the
// status word gets GM_ERR_TIMEOUT and false is returned (the caller returns, so every block
// leaves within one more bounded wait).
__device__ bool nl_grid_sync(unsigned *bar, int32_t *status) {
    __shared__ int expired;
    __syncthreads();
    if (threadIdx.x == 0) {
        expired = 0;
        unsigned g, arrived;
        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(bar + 1) : "memory");
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(bar) : "memory");
        if (arrived == gridDim.x - 1) {
            asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(bar) : "memory");
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar + 1) : "memory");
        } else {
            const unsigned long long t0 = nl_clock_ns();
            unsigned now;
            for (;;) {
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(now) : "l"(bar + 1) : "memory");
                if (now != g) break;
                if (nl_clock_ns() - t0 > 1000000000ull) {
                    set_status(status, GM_ERR_TIMEOUT);
                    expired = 1;
                    break;
                }
                __nanosleep(32);
            }
        }
    }
    __syncthreads();
    return expired == 0;
}

__device__ __forceinline__ int floordiv(int v, int n) { return v >= 0 ? v / n : -((-v + n - 1) / n); }

// ------------------------------------------------------------------ block scan helpers
// Exclusive scan of v over the block; *total gets the block sum.
__device__ __forceinline__ int block_exclusive_scan(int v, int *total) {
    __shared__ int warp_sums[NL_WARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    int wpre = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < NL_WARPS; ++w) {
        const int s = warp_sums[w];
        wpre += w < warp ? s : 0;
        tot += s;
    }
    __syncthreads();
    *total = tot;
    return wpre + x - v;
}

__device__ __forceinline__ int block_sum(int v) {
    __shared__ int warp_sums[NL_WARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) warp_sums[warp] = v;
    __syncthreads();
    int tot = 0;
#pragma unroll
    for (int w = 0; w < NL_WARPS; ++w) tot += warp_sums[w];
    __syncthreads();
    return tot;
}

// ------------------------------------------------------------------ setup
// Box checks on the bit patterns (integer compares keep them off the FP64 unit): an entry is
// zero (+0 or -0), or positive (above +0, at most +inf: NaN fails as in a comparison).
__device__ __forceinline__ bool dzero(double v) { return (__double_as_longlong(v) << 1) == 0; }
__device__ __forceinline__ bool dpositive(double v) {
    const long long b = __double_as_longlong(v);
    return b > 0 && b <= 0x7FF0000000000000ll;
}
// Orthorhombic, periodic on every axis, positive edges
__device__ __forceinline__ bool box_supported(const NlArgs &a, int b) {
    const double *C = a.cell + 9 * b;
    const bool ortho = dzero(C[1]) && dzero(C[2]) && dzero(C[3]) && dzero(C[5]) && dzero(C[6]) && dzero(C[7]);
    const bool periodic = a.pbc[3 * b] && a.pbc[3 * b + 1] && a.pbc[3 * b + 2];
    return ortho && periodic && dpositive(C[0]) && dpositive(C[4]) && dpositive(C[8]);
}

// Cell grid of structure b (FP64, fixed operation order).  Returns its number of cells.
// inv3, when given, holds the three reciprocals 1 / L already (computed one per thread).
__device__ int nl_struct_setup(const NlArgs &a, int b, NlStruct &q, const double *inv3 = nullptr) {
    const double *C = a.cell + 9 * b;
    q.a0 = a.atom_ptr[b];
    q.n = a.atom_ptr[b + 1] - q.a0;
    bool ok = box_supported(a, b);
    long long nc[3];
    // Only L and 1/L (the FP64 wrap) need FP64; the grid (cells per axis, cells per length,
    // stencil widths) and the filter band need to be consistent and conservative, and FP32
    // keeps B300's slow FP64 unit off this per-build latency chain.  Cells stay at least
    // r_cut (1 + 1e-5) long, a margin far above the FP32 rounding.
    const float cells_per_len = 1.0f / ((float)a.rc * (1.0f + 1e-5f));
    for (int d = 0; d < 3; ++d) {
        q.L[d] = ok ? C[4 * d] : 1.0;
        q.invL[d] = inv3 ? inv3[d] : 1.0 / q.L[d];
        const float f = floorf((float)q.L[d] * cells_per_len * (1.0f - 1e-6f));
        nc[d] = f < 1.0f ? 1 : (f > 1024.0f ? 1024 : (long long)f);
    }
    const long long limit = q.n > 1 ? q.n : 1;
    while (nc[0] * nc[1] * nc[2] > limit) {
        int am = 0;
        if (nc[1] > nc[am]) am = 1;
        if (nc[2] > nc[am]) am = 2;
        nc[am] -= 1;
    }
    int Kmax = 0;
    float Lmax = 0.0f;
    const float rcf = (float)a.rc;
    for (int d = 0; d < 3; ++d) {
        q.nc[d] = (int)nc[d];
        q.Lf[d] = (float)q.L[d];
        const float ics = (float)nc[d] / q.Lf[d];
        q.inv_cs[d] = (double)ics;
        int K = (int)ceilf(rcf * ics * (1.0f + 1e-6f) + 1e-6f);
        if (K > 100) { ok = false; K = 0; }
        q.K[d] = ok ? K : 0;
        Kmax = K > Kmax ? K : Kmax;
        Lmax = q.Lf[d] > Lmax ? q.Lf[d] : Lmax;
    }
    if (!ok) set_status(a.status, GM_ERR_UNSUPPORTED);
    // FP32 filter error per axis: the roundings of the two wrapped coordinates and of the
    // image offset (each <= 2^-24 L), of the shifted coordinate (<= 2^-24 2L) and of the
    // difference (<= 2^-24 r_cut near the cutoff) stay below 2^-24 L (8 + 4K); the band
    // bounds the resulting r^2 error near r_cut (x 4, and x 1.01 over the FP32 evaluation)
    const float u = 5.9604644775390625e-8f;  // 2^-24
    const float e = u * Lmax * (8.0f + 4.0f * (float)Kmax);
    q.eps2 = 1.01f * (4.0f * (2.0f * 1.7320508f * e * rcf + 3.0f * e * e + 4.0f * u * rcf * rcf)) + 1e-30f;
    return q.nc[0] * q.nc[1] * q.nc[2];
}

// Block 0 builds the per-structure grids and the global cell numbering; every block
// zeroes its share of the scatter slots (the histogram is cleared before the launch).
__device__ void ph_setup(const NlArgs &a, int bid, int nb) {
    if (bid == 0) {
        int carry = 0;
        for (int chunk = 0; chunk < a.B; chunk += NL_THREADS) {
            const int b = chunk + threadIdx.x;
            NlStruct q;
            const int ncell = b < a.B ? nl_struct_setup(a, b, q) : 0;
            int tot;
            const int pre = block_exclusive_scan(ncell, &tot);
            if (b < a.B) {
                q.cell0 = carry + pre;
                a.S[b] = q;
            }
            carry += tot;
        }
        if (threadIdx.x == 0) {
            *a.ncells = carry;
            *a.n_redo = 0;
        }
    }
    for (int c = bid * NL_THREADS + threadIdx.x; c < a.ncmax; c += nb * NL_THREADS) a.cfill[c] = 0;
}

// Small systems: every block derives all per-structure grids itself (shared memory), so
// binning needs no grid barrier after the setup; block 0 also publishes them.
static_assert(256 * sizeof(NlStruct) <= NL_WARPS * 512 * (sizeof(float4) + sizeof(unsigned)),
              "the structures of a small batch must fit in the search's shared memory");
__device__ void ph_setup_local(const NlArgs &a, int bid, NlStruct *Ss) {
    // the 3 B reciprocals 1 / L first, one per thread (FP64 divisions in parallel), into the
    // structures' own slots
    for (int t = threadIdx.x; t < 3 * a.B; t += NL_THREADS) {
        const int b = t / 3, d = t - 3 * b;
        Ss[b].invL[d] = 1.0 / (box_supported(a, b) ? a.cell[9 * b + 4 * d] : 1.0);
    }
    __syncthreads();
    int carry = 0;
    for (int chunk = 0; chunk < a.B; chunk += NL_THREADS) {
        const int b = chunk + threadIdx.x;
        NlStruct q;
        double inv3[3];
        if (b < a.B) {
            inv3[0] = Ss[b].invL[0];
            inv3[1] = Ss[b].invL[1];
            inv3[2] = Ss[b].invL[2];
        }
        const int ncell = b < a.B ? nl_struct_setup(a, b, q, inv3) : 0;
        int tot;
        const int pre = block_exclusive_scan(ncell, &tot);
        if (b < a.B) {
            q.cell0 = carry + pre;
            Ss[b] = q;
            if (bid == 0) a.S[b] = q;
        }
        carry += tot;
    }
    if (bid == 0 && threadIdx.x == 0) {
        *a.ncells = carry;
        *a.n_redo = 0;
    }
    __syncthreads();
}

// Exclusive scan of src[0..n) (n <= NL_SCAN_ONE_BLOCK) into shared memory dst[0..n] by every
// block; block 0 also publishes it (pub[0..n]; n_pairs and the capacity check when given).
__device__ void ph_scan_local(const int32_t *src, int n, int32_t *dst, int bid, int32_t *pub, int64_t cap,
                              int64_t *n_pairs, int32_t *status) {
    int carry = 0;
    for (int s = 0; s < n; s += NL_SCAN_SUB) {
        const int base = s + threadIdx.x * 4;
        int v[4], sum = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = base + k < n ? src[base + k] : 0;
            sum += v[k];
        }
        int tot;
        int pre = carry + block_exclusive_scan(sum, &tot);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (base + k < n) {
                dst[base + k] = pre;
                if (bid == 0) pub[base + k] = pre;
            }
            pre += v[k];
        }
        carry += tot;
    }
    if (threadIdx.x == 0) {
        dst[n] = carry;
        if (bid == 0) {
            pub[n] = carry;
            if (n_pairs) {
                *n_pairs = carry;
                if ((int64_t)carry > cap) set_status(status, GM_ERR_CAPACITY);
            }
        }
    }
    __syncthreads();
}

// ------------------------------------------------------------------ bin
// Wrap of one coordinate; the same correctly rounded sequence as the oracle.  The image
// count m = floor(x / L) needs the floor of the correctly rounded quotient; the product with
// the rounded reciprocal is within a few ulps of it, so its floor is that floor whenever the
// product is more than 1e-9 from an integer (|quotient| < 1e6); otherwise the division decides.
__device__ __forceinline__ double wrap_axis(double x, double L, double invL, int &m_out) {
    const double qa = __dmul_rn(x, invL);
    double m = floor(qa);
    const double fr = qa - m;
    if (!(fr > 1e-9 && fr < 1.0 - 1e-9 && fabs(qa) < 1e6)) m = floor(__ddiv_rn(x, L));
    double xw = __dsub_rn(x, __dmul_rn(m, L));
    if (xw < 0.0) { m -= 1.0; xw = __dsub_rn(x, __dmul_rn(m, L)); }
    if (xw >= L) { m += 1.0; xw = __dsub_rn(x, __dmul_rn(m, L)); }
    if (xw < 0.0 || xw >= L) xw = 0.0;
    m_out = (fabs(m) < 1.0e6) ? (int)m : 0;
    return xw;
}

// Work spread over blocks first: warp w of block bid takes the 32-atom chunks
// bid + nb (w + 8 k), so a small system occupies many SMs.
__device__ void ph_bin(const NlArgs &a, int bid, int nb, const NlStruct *S) {
    const int lane = threadIdx.x & 31;
    for (int ch = bid + nb * (threadIdx.x >> 5); ch * 32 < a.N; ch += nb * NL_WARPS) {
        const int i = ch * 32 + lane;
        if (i >= a.N) continue;
        const int b = structure_of(a.atom_ptr, a.B, i);
        const int z = a.species[i];
        if (z < 0 || z >= a.n_species) set_status(a.status, GM_ERR_SPECIES);
        const NlStruct &q = S[b];
        int ic[3];
        for (int d = 0; d < 3; ++d) {
            const double x = a.pos[3 * i + d];
            int m;
            const double w = wrap_axis(x, q.L[d], q.invL[d], m);
            if (!(fabs(x) < 1.0e6 * q.L[d])) set_status(a.status, GM_ERR_UNSUPPORTED);
            a.xw[3 * i + d] = w;
            a.mimg[3 * i + d] = m;
            int c = (int)floor(w * q.inv_cs[d]);
            c = c < 0 ? 0 : (c >= q.nc[d] ? q.nc[d] - 1 : c);
            ic[d] = c;
        }
        const int cid = q.cell0 + (ic[2] * q.nc[1] + ic[1]) * q.nc[0] + ic[0];
        a.cellid[i] = cid;
        a.mpk[i] = bytes3(a.mimg[3 * i], a.mimg[3 * i + 1], a.mimg[3 * i + 2]);
        atomicAdd(a.ccount + cid, 1);
    }
    // cell -> structure table for the search passes
    for (int b = bid; b < a.B; b += nb) {
        const NlStruct &q = S[b];
        const int ncb = q.nc[0] * q.nc[1] * q.nc[2];
        for (int c = threadIdx.x; c < ncb; c += NL_THREADS) a.cstruct[q.cell0 + c] = b;
    }
}

// ------------------------------------------------------------------ scan
// Exclusive scan of src[0..n) into dst[0..n] (dst[n] = total) by nb blocks: phase 1 scans
// the blocks' chunks and records their sums, phase 2 adds the sums of the earlier chunks.
__device__ void ph_scan1(const int32_t *src, int32_t *dst, int n, int32_t *bsum, int bid, int nb) {
    const int chunk = (n + nb - 1) / nb;
    const int c0 = min(n, bid * chunk), c1 = min(n, c0 + chunk);
    int carry = 0;
    for (int s = c0; s < c1; s += NL_SCAN_SUB) {
        const int base = s + threadIdx.x * 4;
        int v[4], sum = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = base + k < c1 ? src[base + k] : 0;
            sum += v[k];
        }
        int tot;
        int pre = carry + block_exclusive_scan(sum, &tot);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (base + k < c1) dst[base + k] = pre;
            pre += v[k];
        }
        carry += tot;
    }
    if (threadIdx.x == 0) bsum[bid] = carry;
}

__device__ void ph_scan2(int32_t *dst, int n, const int32_t *bsum, int bid, int nb, int64_t cap, int64_t *n_pairs,
                         int32_t *status) {
    int part = 0;
    for (int k = threadIdx.x; k < bid; k += NL_THREADS) part += bsum[k];
    const int off = block_sum(part);
    const int chunk = (n + nb - 1) / nb;
    const int c0 = min(n, bid * chunk), c1 = min(n, c0 + chunk);
    if (off != 0)
        for (int k = c0 + threadIdx.x; k < c1; k += NL_THREADS) dst[k] += off;
    if (bid == nb - 1 && threadIdx.x == 0) {
        const int total = off + bsum[bid];
        dst[n] = total;
        if (n_pairs) {
            *n_pairs = total;
            if ((int64_t)total > cap) set_status(status, GM_ERR_CAPACITY);
        }
    }
}

// Exclusive scan of src[0..n) into dst[0..n] by block 0 alone (n small).
__device__ void ph_scan_one(const int32_t *src, int32_t *dst, int n, int bid, int64_t cap, int64_t *n_pairs,
                            int32_t *status) {
    if (bid != 0) return;
    int carry = 0;
    for (int s = 0; s < n; s += NL_SCAN_SUB) {
        const int base = s + threadIdx.x * 4;
        int v[4], sum = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = base + k < n ? src[base + k] : 0;
            sum += v[k];
        }
        int tot;
        int pre = carry + block_exclusive_scan(sum, &tot);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (base + k < n) dst[base + k] = pre;
            pre += v[k];
        }
        carry += tot;
    }
    if (threadIdx.x == 0) {
        dst[n] = carry;
        if (n_pairs) {
            *n_pairs = carry;
            if ((int64_t)carry > cap) set_status(status, GM_ERR_CAPACITY);
        }
    }
}

// ------------------------------------------------------------------ scatter and sort
__device__ void ph_scatter(const NlArgs &a, int bid, int nb, const int32_t *cstart) {
    const int lane = threadIdx.x & 31;
    for (int ch = bid + nb * (threadIdx.x >> 5); ch * 32 < a.N; ch += nb * NL_WARPS) {
        const int i = ch * 32 + lane;
        if (i >= a.N) continue;
        const int c = a.cellid[i];
        const int slot = atomicAdd(a.cfill + c, 1);
        a.unsorted[cstart[c] + slot] = i;
    }
}

// One warp per cell: each atom's position in the cell is its rank among the cell's atom
// indices (all distinct), so the packed order is ascending atom index (deterministic).
__device__ void ph_sort(const NlArgs &a, int bid, int nb) {
    const int lane = threadIdx.x & 31;
    const int ncells = *a.ncells;
    for (int c = bid + nb * (threadIdx.x >> 5); c < ncells; c += nb * NL_WARPS) {
        const int s0 = a.cstart[c], n = a.cstart[c + 1] - s0;
        for (int e = lane; e < n; e += 32) {
            const int v = a.unsorted[s0 + e];
            int r = 0;
            for (int k = 0; k < n; ++k) r += a.unsorted[s0 + k] < v;
            a.xs[s0 + r] = make_float4((float)a.xw[3 * v], (float)a.xw[3 * v + 1], (float)a.xw[3 * v + 2],
                                       __int_as_float(v));
            a.xsm[s0 + r] = a.mpk[v];
        }
    }
}

// ------------------------------------------------------------------ search
// Exact FP64 membership test of candidate j of centre i under the image (nx, ny, nz).  Kept
// out of line and reached through a warp vote, so that the rare test is a real branch and
// not predicated FP64 code issued with every candidate test (B300 issues FP64 at a small
// fraction of the FP32 rate).
__device__ __noinline__ bool exact_inside(const double *__restrict__ xw, int j, double xi0, double xi1, double xi2,
                                             int nx, int ny, int nz, const NlStruct &q, double rc2) {
    const double d0 = __dadd_rn(__dsub_rn(xw[3 * j], xi0), __dmul_rn((double)nx, q.L[0]));
    const double d1 = __dadd_rn(__dsub_rn(xw[3 * j + 1], xi1), __dmul_rn((double)ny, q.L[1]));
    const double d2 = __dadd_rn(__dsub_rn(xw[3 * j + 2], xi2), __dmul_rn((double)nz, q.L[2]));
    return __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2)) < rc2;
}

// Store pair (i, j) with its lattice shift relative to the caller's (unwrapped) positions:
// image n of the wrapped positions minus the image counts of j, plus those of i.
__device__ __forceinline__ void store_pair(const NlArgs &a, int pos, int j, int s0, int s1, int s2) {
    if (s0 < -127 || s0 > 127 || s1 < -127 || s1 > 127 || s2 < -127 || s2 > 127) set_status(a.status, GM_ERR_UNSUPPORTED);
    a.col[pos] = j;
    a.shift[pos] = make_char4((signed char)s0, (signed char)s1, (signed char)s2, 0);
}

// Per-atom search over the full stencil (any K): one warp, 32 candidates of a cell per step.
template <bool FILL>
__device__ void search_atom_generic(const NlArgs &a, const NlStruct &q, int c_local, float4 me, int lane,
                                    int row_start = 0) {
    const int i = __float_as_int(me.w);
    const int ix = c_local % q.nc[0], iy = (c_local / q.nc[0]) % q.nc[1], iz = c_local / (q.nc[0] * q.nc[1]);
    const double rc2 = __dmul_rn(a.rc, a.rc);
    const float lo = a.rc2f - q.eps2, hi = a.rc2f + q.eps2;
    const int mi0 = a.mimg[3 * i], mi1 = a.mimg[3 * i + 1], mi2 = a.mimg[3 * i + 2];
    const double xi0 = a.xw[3 * i], xi1 = a.xw[3 * i + 1], xi2 = a.xw[3 * i + 2];
    const unsigned below = (1u << lane) - 1u;
    int out = FILL ? row_start : 0;
    int cnt = 0;
    for (int dz = -q.K[2]; dz <= q.K[2]; ++dz) {
        const int vz = iz + dz, nz = floordiv(vz, q.nc[2]), cz = vz - nz * q.nc[2];
        for (int dy = -q.K[1]; dy <= q.K[1]; ++dy) {
            const int vy = iy + dy, ny = floordiv(vy, q.nc[1]), cy = vy - ny * q.nc[1];
            for (int dx = -q.K[0]; dx <= q.K[0]; ++dx) {
                const int vx = ix + dx, nx = floordiv(vx, q.nc[0]), cx = vx - nx * q.nc[0];
                const int c = q.cell0 + (cz * q.nc[1] + cy) * q.nc[0] + cx;
                const float sx = (float)nx * q.Lf[0], sy = (float)ny * q.Lf[1], sz = (float)nz * q.Lf[2];
                const bool zero_shift = (nx | ny | nz) == 0;
                const int k0 = a.cstart[c], k1 = a.cstart[c + 1];
                for (int base = k0; base < k1; base += 32) {
                    const int k = base + lane;
                    bool in = false, band = false;
                    int j = 0;
                    if (k < k1) {
                        const float4 o = a.xs[k];
                        j = __float_as_int(o.w);
                        if (!(zero_shift && j == i)) {
                            const float fx = (o.x + sx) - me.x, fy = (o.y + sy) - me.y, fz = (o.z + sz) - me.z;
                            const float r2 = fx * fx + fy * fy + fz * fz;
                            in = r2 < lo;
                            band = !in && r2 <= hi;
                        }
                    }
                    if (__any_sync(0xffffffffu, band)) {
                        if (band) in = exact_inside(a.xw, j, xi0, xi1, xi2, nx, ny, nz, q, rc2);
                    }
                    const unsigned ball = __ballot_sync(0xffffffffu, in);
                    if (FILL) {
                        if (in)
                            store_pair(a, out + __popc(ball & below), j, nx - a.mimg[3 * j] + mi0,
                                       ny - a.mimg[3 * j + 1] + mi1, nz - a.mimg[3 * j + 2] + mi2);
                        out += __popc(ball);
                    } else {
                        cnt += __popc(ball);
                    }
                }
            }
        }
    }
    if (!FILL && lane == 0) a.counts[i] = cnt;
}

// Search passes.  SM_SLAB (the default) tests every candidate once and appends the accepted
// ones, with their lattice shifts, to the home atom's slab row (up to maxn; the count is exact
// either way); the compaction then copies the rows into the CSR list.  SM_COUNT and SM_FILL
// are the two-pass alternative for a workspace without the slab (count, then write the CSR
// rows directly once the offsets are known).
//
// One warp per work item = (cell, part): part p of `split` takes the home atoms p, p + split,
// ... of the cell, up to 32 at a time (FP32 positions and indices in shared memory, broadcast
// to the lanes).  Lane t < 27 holds stencil cell t (first sorted index, count, image).  The
// warp stages up to NL_WIN candidates at a time in its own slice of shared memory -- every
// lane issues its loads before storing, each candidate finding its stencil cell by a binary
// search over the lanes' offsets -- and tests 32 staged candidates at a time against every
// home atom.  Only chunks that hold candidates of the home cell itself check for the (i, i,
// n = 0) self pair.  A candidate's info word holds its stencil cell (bits 0..4) and, for the
// writing passes, its image minus its own image counts as bytes3 (bits 8..31, NL_FAR-style
// flag in bit 5); the pair's shift adds the home atom's image counts.
enum SearchMode { SM_COUNT, SM_FILL, SM_SLAB };
constexpr int NL_WIN = 512;
constexpr int NL_STAGE_UNROLL = 8;
// dynamic shared memory of the search passes: staged candidates, their info words, and
// each warp's home atoms
constexpr size_t NL_SMEM = (size_t)NL_WARPS * NL_WIN * (sizeof(float4) + sizeof(unsigned)) + NL_WARPS * 32 * sizeof(float4);
__device__ __forceinline__ float4 *nl_home_smem(float4 *smem) {
    return reinterpret_cast<float4 *>(reinterpret_cast<unsigned *>(smem + NL_WARPS * NL_WIN) + NL_WARPS * NL_WIN);
}

// lattice shift of pair (i, j) with image (n0, n1, n2), from the full image counts
__device__ __forceinline__ unsigned shift_slow(const NlArgs &a, int i, int j, int n0, int n1, int n2) {
    const int s0 = n0 - a.mimg[3 * j] + a.mimg[3 * i];
    const int s1 = n1 - a.mimg[3 * j + 1] + a.mimg[3 * i + 1];
    const int s2 = n2 - a.mimg[3 * j + 2] + a.mimg[3 * i + 2];
    return bytes3(s0, s1, s2);
}

// The tests of one chunk (32 staged candidates, one per lane) against the ng home atoms,
// four home atoms at a time: their distance tests, ballots and row offsets are independent
// chains, and the rare exact FP64 test is one vote per four home atoms (one home atom per
// step left each warp waiting on its own vote -> shuffle -> store chain).  The pairs land
// in the same slots as one home atom at a time.
// UNI: all home atoms of the group have the same image counts, so the staged info word
// already holds the pair's complete shift.
template <int MODE, bool SELF, bool UNI>
__device__ __forceinline__ void test_chunk(const NlArgs &a, const float4 *home, int ng, float4 cv, bool valid, int j,
                                           unsigned info, int n0, int n1, int n2, float lo2, float hi2,
                                           const NlStruct &q, double rc2, int lane, int &hacc, unsigned hmb,
                                           bool &hredo) {
    constexpr int G = 4;
    const unsigned full = 0xffffffffu, below = (1u << lane) - 1u;
    const int st = (int)(info & 31u);
    const int selfj = (SELF && valid && st == NL_HOME_STENCIL) ? j : -1;
    const unsigned vb = (info & 32u) ? NL_FAR : (info >> 8);
    // slab entry of a uniform group (shift complete at staging)
    const unsigned ucode = (MODE == SM_SLAB && UNI) ? shift_code(vb) : 0u;
    const bool maybe_nocode = MODE == SM_SLAB && (!UNI || __any_sync(full, valid && ucode == NL_NOCODE));
    for (int h0 = 0; h0 < ng; h0 += G) {                 // ng <= 32, so h0 + G - 1 <= 31
        bool in[G], band[G];
        int hi[G];
        bool anyband = false;
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const int h = h0 + k;
            const float4 hv = home[h < ng ? h : h0];
            hi[k] = __float_as_int(hv.w);
            const float fx = cv.x - hv.x, fy = cv.y - hv.y, fz = cv.z - hv.z;
            const float r2 = fx * fx + fy * fy + fz * fz;
            const bool other = h < ng && (SELF ? (valid && selfj != hi[k]) : valid);
            in[k] = other && r2 < lo2;
            band[k] = other && !in[k] && r2 <= hi2;      // inside the band: exact FP64 test
            anyband |= band[k];
        }
        if (__any_sync(full, anyband)) {
#pragma unroll
            for (int k = 0; k < G; ++k)
                if (band[k])
                    in[k] = exact_inside(a.xw, j, a.xw[3 * hi[k]], a.xw[3 * hi[k] + 1], a.xw[3 * hi[k] + 2], n0, n1,
                                         n2, q, rc2);
        }
        unsigned ball[G];
#pragma unroll
        for (int k = 0; k < G; ++k) ball[k] = __ballot_sync(full, in[k]);
        if (MODE != SM_COUNT) {
            int ob[G];
            unsigned mb[G];
#pragma unroll
            for (int k = 0; k < G; ++k) {
                ob[k] = __shfl_sync(full, hacc, h0 + k);
                mb[k] = UNI ? 0u : __shfl_sync(full, hmb, h0 + k);
            }
            bool nocode[G];
#pragma unroll
            for (int k = 0; k < G; ++k) {
                nocode[k] = false;
                if (in[k]) {
                    const int pos = ob[k] + __popc(ball[k] & below);
                    if (MODE == SM_SLAB) {
                        const unsigned code = UNI ? ucode : shift_code(bytes3_add(vb, mb[k]));
                        nocode[k] = code == NL_NOCODE;
                        if (pos < a.maxn) a.slab[(size_t)hi[k] * a.maxn + pos] = (unsigned)j | (code << 27);
                    } else {
                        unsigned sh = UNI ? vb : bytes3_add(vb, mb[k]);
                        if (sh & NL_FAR) sh = shift_slow(a, hi[k], j, n0, n1, n2);
                        if (sh & NL_FAR) {
                            set_status(a.status, GM_ERR_UNSUPPORTED);
                            sh = 0;
                        }
                        a.col[pos] = j;
                        reinterpret_cast<unsigned *>(a.shift)[pos] = sh;
                    }
                }
            }
            if (maybe_nocode) {
#pragma unroll
                for (int k = 0; k < G; ++k)
                    if (__any_sync(full, nocode[k]) && lane == h0 + k) hredo = true;
            }
        }
#pragma unroll
        for (int k = 0; k < G; ++k)
            if (lane == h0 + k) hacc += __popc(ball[k]);
    }
}

// Mark row i for the per-atom search during the compaction.
__device__ __forceinline__ void nl_redo(const NlArgs &a, int i) {
    a.redo[i] = 1;
    const int r = atomicAdd(a.n_redo, 1);
    if (r < a.N) a.redo_list[r] = i;
    else set_status(a.status, GM_ERR_ARG);
}

template <int MODE>
__device__ void ph_search(const NlArgs &a, int bid, int nb, float4 *smem) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4 *s_home = nl_home_smem(smem) + 32 * warp;
    float4 *wc = smem + warp * NL_WIN;
    unsigned *wi = reinterpret_cast<unsigned *>(smem + NL_WARPS * NL_WIN) + warp * NL_WIN;
    const unsigned full = 0xffffffffu;
    if (MODE == SM_FILL && __shfl_sync(full, lane == 0 ? (int)status_bad(a.status) : 0, 0)) return;
    // items are claimed from a counter (one per pass): a fixed deal of 2-3 items per warp left
    // most warps waiting at the next grid barrier for the ones with one item more.  The last
    // cells (about one item per warp of the grid) are cut into twice as many parts, so the
    // final round of claims is half as long
    const int ncells = *a.ncells, s1 = a.split, s2 = 2 * s1;
    const int xt = min(ncells, max(1, nb * NL_WARPS / s2));       // cells cut finer
    const int head = (ncells - xt) * s1;
    const int items = head + xt * s2;
    const double rc2 = __dmul_rn(a.rc, a.rc);
    int32_t *ctr = a.item_ctr + (MODE == SM_FILL ? 1 : 0);
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(ctr, 1);
        it = __shfl_sync(full, it, 0);
        if (it >= items) break;
        const int sp = it < head ? s1 : s2;                       // parts of this item's cell
        const int c = it < head ? it / s1 : ncells - xt + (it - head) / s2;
        const int part = it < head ? it - c * s1 : (it - head) % s2;
        const int h0 = a.cstart[c], nh = a.cstart[c + 1] - h0;
        if (part >= nh) continue;                                  // uniform over the warp
        const NlStruct &q = a.S[a.cstruct[c]];
        const int cl = c - q.cell0;
        if (!(q.K[0] == 1 && q.K[1] == 1 && q.K[2] == 1)) {
            // several images per stencil direction: per-atom search (with a slab, the
            // compaction writes these rows with the same routine)
            for (int h = part; h < nh; h += sp) {
                const float4 me = a.xs[h0 + h];
                if (MODE == SM_FILL) {
                    search_atom_generic<true>(a, q, cl, me, lane, a.row_ptr[__float_as_int(me.w)]);
                } else {
                    search_atom_generic<false>(a, q, cl, me, lane);
                    if (MODE == SM_SLAB && lane == 0) nl_redo(a, __float_as_int(me.w));
                }
            }
            continue;
        }
        int k0 = 0, cnt = 0;
        unsigned npk = 0;
        float shx = 0.0f, shy = 0.0f, shz = 0.0f;
        if (lane < 27) {
            const int dz = lane / 9 - 1, dy = (lane / 3) % 3 - 1, dx = lane % 3 - 1;
            const int ix = cl % q.nc[0], iy = (cl / q.nc[0]) % q.nc[1], iz = cl / (q.nc[0] * q.nc[1]);
            const int vz = iz + dz, nz = floordiv(vz, q.nc[2]), cz = vz - nz * q.nc[2];
            const int vy = iy + dy, ny = floordiv(vy, q.nc[1]), cy = vy - ny * q.nc[1];
            const int vx = ix + dx, nx = floordiv(vx, q.nc[0]), cx = vx - nx * q.nc[0];
            const int cc = q.cell0 + (cz * q.nc[1] + cy) * q.nc[0] + cx;
            k0 = a.cstart[cc];
            cnt = a.cstart[cc + 1] - k0;
            npk = bytes3(nx, ny, nz);
            shx = (float)nx * q.Lf[0];
            shy = (float)ny * q.Lf[1];
            shz = (float)nz * q.Lf[2];
        }
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(full, incl, o);
            if (lane >= o) incl += y;
        }
        const int off = incl - cnt;                                // first candidate of stencil cell `lane`
        const int T = __shfl_sync(full, incl, 26);
        const int home_lo = __shfl_sync(full, off, NL_HOME_STENCIL);
        const int home_hi = home_lo + __shfl_sync(full, cnt, NL_HOME_STENCIL);
        const float lo2 = a.rc2f - q.eps2, hi2 = a.rc2f + q.eps2;
        const int nhp = (nh - part + sp - 1) / sp;                 // home atoms of the item
        for (int g0 = 0; g0 < nhp; g0 += 32) {
            const int ng = min(32, nhp - g0);
            int hidx = 0, hacc = 0;
            unsigned hmb = 0;
            bool hredo = false;
            if (lane < ng) {
                const int hk = h0 + part + sp * (g0 + lane);
                const float4 hv = a.xs[hk];
                hidx = __float_as_int(hv.w);
                s_home[lane] = hv;
                if (MODE != SM_COUNT) hmb = a.xsm[hk];
                if (MODE == SM_FILL) hacc = a.row_ptr[hidx];
            }
            // one image count for the whole group (the usual case): shifts complete at staging
            const unsigned m_first = __shfl_sync(full, hmb, 0);
            const bool uni = MODE == SM_COUNT ||
                             (__all_sync(full, lane >= ng || hmb == m_first) && !(m_first & NL_FAR));
            for (int w0 = 0; w0 < T; w0 += NL_WIN) {
                const int wn = min(NL_WIN, T - w0);
                __syncwarp();
                // stage candidates w0 .. w0 + wn: loads first, then the stores
                for (int u0 = 0; u0 < wn; u0 += 32 * NL_STAGE_UNROLL) {
                    float4 o[NL_STAGE_UNROLL];
                    unsigned pm[NL_STAGE_UNROLL];
                    int sts[NL_STAGE_UNROLL];
#pragma unroll
                    for (int u = 0; u < NL_STAGE_UNROLL; ++u) {
                        const int e = w0 + u0 + 32 * u + lane;
                        int st = 0;
#pragma unroll
                        for (int step = 16; step > 0; step >>= 1) {
                            const int t = st + step;
                            const int ot = __shfl_sync(full, off, t & 31);
                            if (t <= 26 && ot <= e) st = t;
                        }
                        const int kc = __shfl_sync(full, k0, st) + (e - __shfl_sync(full, off, st));
                        sts[u] = st;
                        o[u] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                        pm[u] = 0;
                        if (e < w0 + wn) {
                            o[u] = a.xs[kc];
                            if (MODE != SM_COUNT) pm[u] = a.xsm[kc];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < NL_STAGE_UNROLL; ++u) {
                        const int el = u0 + 32 * u + lane;
                        const int st = sts[u];
                        const float sx = __shfl_sync(full, shx, st), sy = __shfl_sync(full, shy, st),
                                    sz = __shfl_sync(full, shz, st);
                        unsigned info = (unsigned)st;
                        if (MODE != SM_COUNT) {
                            // image minus the neighbour's image counts (plus the group's own, if uniform)
                            const unsigned n = __shfl_sync(full, npk, st);
                            const unsigned mh = uni ? m_first : 0u;
                            const unsigned v = (pm[u] & NL_FAR)
                                                   ? NL_FAR
                                                   : bytes3(byte_at(n, 0) - byte_at(pm[u], 0) + byte_at(mh, 0),
                                                            byte_at(n, 1) - byte_at(pm[u], 1) + byte_at(mh, 1),
                                                            byte_at(n, 2) - byte_at(pm[u], 2) + byte_at(mh, 2));
                            info |= (v & NL_FAR) ? 32u : (v << 8);
                        }
                        if (el < wn) {
                            wc[el] = make_float4(o[u].x + sx, o[u].y + sy, o[u].z + sz, o[u].w);
                            wi[el] = info;
                        }
                    }
                }
                __syncwarp();
                for (int base = 0; base < wn; base += 32) {
                    const int el = base + lane;
                    const bool valid = el < wn;
                    float4 cv = make_float4(3.0e30f, 3.0e30f, 3.0e30f, 0.0f);
                    unsigned info = 0;
                    if (valid) {
                        cv = wc[el];
                        info = wi[el];
                    }
                    const int j = __float_as_int(cv.w);
                    const unsigned n = __shfl_sync(full, npk, (int)(info & 31u));
                    const int n0 = byte_at(n, 0), n1 = byte_at(n, 1), n2 = byte_at(n, 2);
                    // does the chunk overlap the home cell's candidates?
                    const int e0 = w0 + base;
                    const bool self = e0 < home_hi && e0 + 32 > home_lo;
                    if (uni) {
                        if (self)
                            test_chunk<MODE, true, true>(a, s_home, ng, cv, valid, j, info, n0, n1, n2, lo2, hi2,
                                                         q, rc2, lane, hacc, hmb, hredo);
                        else
                            test_chunk<MODE, false, true>(a, s_home, ng, cv, valid, j, info, n0, n1, n2, lo2, hi2,
                                                          q, rc2, lane, hacc, hmb, hredo);
                    } else if (MODE != SM_COUNT) {
                        test_chunk<MODE, true, false>(a, s_home, ng, cv, valid, j, info, n0, n1, n2, lo2, hi2, q,
                                                      rc2, lane, hacc, hmb, hredo);
                    }
                }
            }
            if (MODE != SM_FILL && lane < ng) {
                a.counts[hidx] = hacc;
                if (MODE == SM_SLAB) {
                    const bool over = hacc > a.maxn || hredo;
                    a.redo[hidx] = over ? 1 : 0;
                    if (over) nl_redo(a, hidx);
                }
            }
            __syncwarp();                                              // s_home is rewritten next
        }
    }
}

// stencil cell (0..26) of staged candidate e, from the cells' exclusive offsets off[0..27]
__device__ __forceinline__ int stencil_of(int e, const int *off) {
    int st = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const int t = st + step;
        if (t <= 26 && off[t] <= e) st = t;
    }
    return st;
}

// Block-level variant of the search passes (small systems, where the warp-level one leaves
// most of the GPU idle and restages the same candidates for every part of a cell): a work
// item = (cell, part) per block; warp 0 builds the stencil, all 256 threads stage the item's
// candidates (up to NL_BCAND) once, and warp w takes the home atoms part + split (w + 8 r).
// The image counts are folded into the staged shifts when they agree over the item's home
// atoms.  Items with more candidates than fit take the per-atom search.
constexpr int NL_BCAND = NL_WARPS * NL_WIN;

// Items are claimed from a counter (one per pass) rather than dealt in a fixed order: item
// costs vary by an order of magnitude over a batch of boxes of different sizes, and a fixed
// deal left the slowest block at twice the mean.  Thread 0 claims the next item while the
// block works on the current one.
template <int MODE>
__device__ void ph_search_block(const NlArgs &a, int bid, int nb, float4 *smem) {
    __shared__ int s_k0[27], s_off[28];
    __shared__ unsigned s_n[27];
    __shared__ float s_sh[27][3];
    __shared__ int s_skip, s_item;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4 *cand = smem;
    unsigned *cinfo = reinterpret_cast<unsigned *>(smem + NL_BCAND);
    const unsigned full = 0xffffffffu, below = (1u << lane) - 1u;
    if (threadIdx.x == 0) s_skip = MODE == SM_FILL && status_bad(a.status);
    __syncthreads();
    if (s_skip) return;                                            // uniform over the block
    const int items = *a.ncells * a.split;
    const double rc2 = __dmul_rn(a.rc, a.rc);
    int32_t *ctr = a.item_ctr + (MODE == SM_FILL ? 1 : 0);
    if (threadIdx.x == 0) s_item = atomicAdd(ctr, 1);
    __syncthreads();
    for (int it = s_item; it < items; it = s_item) {
        int next = 0;
        if (threadIdx.x == 0) next = atomicAdd(ctr, 1);           // consumed at the end of the item
        const int c = it / a.split, part = it - c * a.split;
        const int h0 = a.cstart[c], nh = a.cstart[c + 1] - h0;
        const NlStruct &q = a.S[a.cstruct[c]];
        const int cl = c - q.cell0;
        const bool tiled = q.K[0] == 1 && q.K[1] == 1 && q.K[2] == 1;
        if (part >= nh) {                                          // uniform over the block
            __syncthreads();
            if (threadIdx.x == 0) s_item = next;
            __syncthreads();
            continue;
        }
        int T = 0;
        if (tiled) {
            if (warp == 0) {
                int k0 = 0, cnt = 0;
                if (lane < 27) {
                    const int dz = lane / 9 - 1, dy = (lane / 3) % 3 - 1, dx = lane % 3 - 1;
                    const int ix = cl % q.nc[0], iy = (cl / q.nc[0]) % q.nc[1], iz = cl / (q.nc[0] * q.nc[1]);
                    const int vz = iz + dz, nz = floordiv(vz, q.nc[2]), cz = vz - nz * q.nc[2];
                    const int vy = iy + dy, ny = floordiv(vy, q.nc[1]), cy = vy - ny * q.nc[1];
                    const int vx = ix + dx, nx = floordiv(vx, q.nc[0]), cx = vx - nx * q.nc[0];
                    const int cc = q.cell0 + (cz * q.nc[1] + cy) * q.nc[0] + cx;
                    k0 = a.cstart[cc];
                    cnt = a.cstart[cc + 1] - k0;
                    s_k0[lane] = k0;
                    s_n[lane] = bytes3(nx, ny, nz);
                    s_sh[lane][0] = (float)nx * q.Lf[0];
                    s_sh[lane][1] = (float)ny * q.Lf[1];
                    s_sh[lane][2] = (float)nz * q.Lf[2];
                }
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(full, incl, o);
                    if (lane >= o) incl += y;
                }
                if (lane < 27) s_off[lane + 1] = incl;
                if (lane == 0) s_off[0] = 0;
            }
            __syncthreads();
            T = s_off[27];
        }
        // image counts common to all home atoms of the item?
        unsigned m_first = 0;
        bool uni = true;
        if (MODE != SM_COUNT) {
            m_first = a.xsm[h0 + part];
            bool same = true;
            for (int h = part + a.split * threadIdx.x; h < nh; h += a.split * NL_THREADS) same &= a.xsm[h0 + h] == m_first;
            uni = __syncthreads_and(same) && !(m_first & NL_FAR);
        }
        if (!tiled || T > NL_BCAND) {
            for (int h = part + a.split * warp; h < nh; h += a.split * NL_WARPS) {
                const float4 me = a.xs[h0 + h];
                if (MODE == SM_FILL) {
                    search_atom_generic<true>(a, q, cl, me, lane, a.row_ptr[__float_as_int(me.w)]);
                } else {
                    search_atom_generic<false>(a, q, cl, me, lane);
                    if (MODE == SM_SLAB && lane == 0) nl_redo(a, __float_as_int(me.w));
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) s_item = next;
            __syncthreads();
            continue;
        }
        // stage all candidates of the item (loads before stores), then pad to a multiple of
        // 32 with far-away dummies (no bounds test in the chunk loop)
        bool nocode_seen = false;
        for (int e0 = threadIdx.x; e0 < T; e0 += NL_THREADS * 4) {
            float4 o[4];
            unsigned pm[4];
            int sts[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + NL_THREADS * u;
                int st = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int t = st + step;
                    if (t <= 26 && s_off[t] <= e) st = t;
                }
                sts[u] = st;
                o[u] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                pm[u] = 0;
                if (e < T) {
                    const int kc = s_k0[st] + (e - s_off[st]);
                    o[u] = a.xs[kc];
                    if (MODE != SM_COUNT) pm[u] = a.xsm[kc];
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + NL_THREADS * u;
                if (e < T) {
                    const int st = sts[u];
                    unsigned info = (unsigned)st;
                    if (MODE != SM_COUNT) {
                        const unsigned n = s_n[st], mh = uni ? m_first : 0u;
                        const unsigned v = (pm[u] & NL_FAR) ? NL_FAR
                                                            : bytes3(byte_at(n, 0) - byte_at(pm[u], 0) + byte_at(mh, 0),
                                                                     byte_at(n, 1) - byte_at(pm[u], 1) + byte_at(mh, 1),
                                                                     byte_at(n, 2) - byte_at(pm[u], 2) + byte_at(mh, 2));
                        info |= (v & NL_FAR) ? 32u : (v << 8);
                    }
                    cand[e] = make_float4(o[u].x + s_sh[st][0], o[u].y + s_sh[st][1], o[u].z + s_sh[st][2], o[u].w);
                    // uniform single-pass items stage the complete slab entry (index | shift code)
                    if (MODE == SM_SLAB && uni) {
                        const unsigned code = shift_code((info & 32u) ? NL_FAR : (info >> 8));
                        nocode_seen |= code == NL_NOCODE;
                        info = (unsigned)__float_as_int(o[u].w) | (code << 27);
                    }
                    cinfo[e] = info;
                }
            }
        }
        const int Tp = (T + 31) & ~31;
        if (threadIdx.x < Tp - T) {
            cand[T + threadIdx.x] = make_float4(3.0e30f, 3.0e30f, 3.0e30f, 0.0f);
            cinfo[T + threadIdx.x] = 0u;
        }
        // rows that meet a shift outside {-1, 0, 1}^3 need the redo; uniform items know it here
        const bool check_codes = MODE == SM_SLAB && (!uni || __syncthreads_or(nocode_seen));
        __syncthreads();
        const int home_lo = s_off[NL_HOME_STENCIL];
        const float lo2 = a.rc2f - q.eps2, hi2 = a.rc2f + q.eps2;
        const int nhp = (nh - part + a.split - 1) / a.split;       // home atoms of the item
        // Warp w takes home atoms r = w, w + 8, ... of the item, one at a time against all T
        // candidates in chunks of 32: the row offset is a warp-uniform register and the home
        // position is the staged copy from the home stencil cell (shift 0), so the chunk loop
        // has no shuffles and no global loads.
        for (int r = warp; r < nhp; r += NL_WARPS) {
            const int hl = part + a.split * r;                     // index within the home cell
            const int self_e = home_lo + hl;                       // the home atom's own staged copy
            const float4 hv = cand[self_e];
            const int hi = __float_as_int(hv.w);
            const unsigned hmb = (MODE != SM_COUNT && !uni) ? a.xsm[h0 + hl] : 0u;
            const int rb = MODE == SM_FILL ? a.row_ptr[hi] : 0;
            uint32_t *srow = MODE == SM_SLAB ? a.slab + (size_t)hi * a.maxn : nullptr;
            int cnt = 0;
            bool hredo = false;
            for (int base = 0; base < Tp; base += 32) {
                const int e = base + lane;
                const float4 cv = cand[e];
                const unsigned w = cinfo[e];
                const int j = __float_as_int(cv.w);
                const float fx = cv.x - hv.x, fy = cv.y - hv.y, fz = cv.z - hv.z;
                const float r2 = fx * fx + fy * fy + fz * fz;
                const bool other = e != self_e;
                bool in = other && r2 < lo2;
                const bool band = other && !in && r2 <= hi2;          // inside the band: exact FP64 test
                if (__any_sync(full, band)) {
                    if (band) {
                        const unsigned n = s_n[stencil_of(e, s_off)];
                        in = exact_inside(a.xw, j, a.xw[3 * hi], a.xw[3 * hi + 1], a.xw[3 * hi + 2], byte_at(n, 0),
                                          byte_at(n, 1), byte_at(n, 2), q, rc2);
                    }
                }
                const unsigned ball = __ballot_sync(full, in);
                if (MODE != SM_COUNT && in) {
                    const int pos = cnt + __popc(ball & below);
                    const unsigned vb = (w & 32u) ? NL_FAR : (w >> 8);
                    if (MODE == SM_SLAB) {
                        const unsigned ent =
                            uni ? w : ((unsigned)j | (shift_code(bytes3_add(vb, hmb)) << 27));
                        if (check_codes) hredo |= (ent >> 27) == NL_NOCODE;
                        if (pos < a.maxn) srow[pos] = ent;
                    } else {
                        unsigned sh = uni ? vb : bytes3_add(vb, hmb);
                        if (sh & NL_FAR) {
                            const unsigned n = s_n[stencil_of(e, s_off)];
                            sh = shift_slow(a, hi, j, byte_at(n, 0), byte_at(n, 1), byte_at(n, 2));
                        }
                        if (sh & NL_FAR) {
                            set_status(a.status, GM_ERR_UNSUPPORTED);
                            sh = 0;
                        }
                        a.col[rb + pos] = j;
                        reinterpret_cast<unsigned *>(a.shift)[rb + pos] = sh;
                    }
                }
                cnt += __popc(ball);
            }
            if (check_codes) hredo = __any_sync(full, hredo);
            if (MODE != SM_FILL && lane == 0) {
                a.counts[hi] = cnt;
                if (MODE == SM_SLAB) {
                    const bool over = cnt > a.maxn || hredo;
                    a.redo[hi] = over ? 1 : 0;
                    if (over) nl_redo(a, hi);
                }
            }
        }
        __syncthreads();                                           // the staging is rewritten next
        if (threadIdx.x == 0) s_item = next;
        __syncthreads();
    }
}

// ------------------------------------------------------------------ brute-force search
// Structures of at most BR_MAXN atoms whose boxes are at least r_cut long on every axis (one
// stencil cell per axis): a warp tests its atom against every atom of its structure -- no
// histogram, scatter or sort phases.  From 2.001 r_cut each neighbour has exactly one image
// within r_cut (the minimum image); shorter boxes take the multi-image row (brute_row_multi).  The row
// comes out in the cell-list order all the same: with the cell grid of the setup, the
// stencil cell of pair (i, j, n) is d = c_j + n nc - c_i per axis (in {-1, 0, 1}, cells
// being at least r_cut long), and the accepted pairs, found in ascending j, are placed by a
// stable counting sort on that stencil index.  A row longer than BR_CAP (shared memory)
// sends the whole build back to the cell-list path.
//
// A buffered pair is one word: stencil << 27 | image << 22 | j, the image n coded as
// (n_x + 1) + 3 (n_y + 1) + 9 (n_z + 1) and j < 2^22.  The per-atom cell word of the wrap,
// w = c_x + 3 c_y + 9 c_z (an exact small integer in FP32), gives the stencil index
// (s_x + 1) + 3 (s_y + 1) + 9 (s_z + 1) as 13 + w_j - w_i + n . (nc_x, 3 nc_y, 9 nc_z).
constexpr int BR_CAP = 512;
static_assert(GM_MAX_ATOMS <= (1 << 22), "brute-force keys hold the neighbour index in 22 bits");
struct BrBuf {
    unsigned key[BR_CAP];
    unsigned row[BR_CAP];   // the placed row (j | shift code << 27), kept for the direct write
    int hist[32], run[32];
    int rowi, rowcnt;       // the warp's placed row (rowi -1: none)
};

// shared-memory layout of the small-system brute-force path: the per-structure grids (at most
// 256) and the row scan (at most 4097 ints) first, then one buffer per warp
constexpr size_t NL_BR_OFF = ((256 * sizeof(NlStruct) > 4097 * sizeof(int32_t) ? 256 * sizeof(NlStruct)
                                                                               : 4097 * sizeof(int32_t)) + 127) / 128 * 128;
// the row scan of the mid-size brute-force path: N + 1 <= 2 NL_SCAN_ONE_BLOCK entries
static_assert(NL_BR_OFF >= 2 * NL_SCAN_ONE_BLOCK * sizeof(int32_t), "row scan of the mid-size path");
static_assert(NL_BR_OFF + NL_WARPS * sizeof(BrBuf) <= NL_SMEM, "brute-force buffers exceed the search's shared memory");
// the batch path's copy of atom_ptr sits after the row buffers (at most BR_PTR_MAX entries)
constexpr size_t NL_BR_PTR_OFF = NL_BR_OFF + NL_WARPS * sizeof(BrBuf);
constexpr int BR_PTR_MAX = (int)((NL_SMEM - NL_BR_PTR_OFF) / sizeof(int32_t));

// structure of atom i from a copy of atom_ptr (shared or global memory)
__device__ __forceinline__ int structure_in(const int32_t *ptr, int n_struct, int i) {
    int lo = 0, hi = n_struct - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ptr[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// every structure has one stencil cell per axis (box edges at least r_cut: single-image rows
// from 2 r_cut, multi-image rows below) and at most BR_MAXN atoms (the search is quadratic)
constexpr int BR_MAXN = 2048;
__device__ bool nl_brute_eligible(const NlArgs &a, const NlStruct *Ss) {
    bool ok = true;
    for (int b = threadIdx.x; b < a.B; b += blockDim.x) {
        const NlStruct &q = Ss[b];
        ok = ok && q.n <= BR_MAXN;
#pragma unroll
        for (int d = 0; d < 3; ++d) ok = ok && q.K[d] == 1 && q.Lf[d] >= 1.0001f * (float)a.rc;
    }
    return __syncthreads_and(ok);
}

// wrap (as ph_bin) without the histogram; xs[i] = FP32 wrapped position with the cell word
// c_x + 3 c_y + 9 c_z (as a float) in w, indexed by atom.  One lane per axis (ten atoms per
// warp, lanes 30 and 31 idle): the FP64 wrap of an atom runs on three lanes at once, and its
// axis-0 lane gathers the other two by shuffles.
__device__ void ph_wrap_brute(const NlArgs &a, int bid, int nb, const NlStruct *S, const int32_t *sptr = nullptr) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, ga = lane / 3, d = lane - 3 * ga;
    const int l1 = min(3 * ga + 1, 31), l2 = min(3 * ga + 2, 31);
    for (int g = bid + nb * (threadIdx.x >> 5); g * 10 < a.N; g += nb * NL_WARPS) {
        const int i = g * 10 + ga;
        const bool act = lane < 30 && i < a.N;
        float wf = 0.0f;
        int c = 0;
        if (act) {
            const NlStruct &q = S[sptr ? structure_in(sptr, a.B, i) : structure_of(a.atom_ptr, a.B, i)];
            if (d == 0) {
                const int z = a.species[i];
                if (z < 0 || z >= a.n_species) set_status(a.status, GM_ERR_SPECIES);
            }
            const double x = a.pos[3 * i + d];
            int m;
            const double w = wrap_axis(x, q.L[d], q.invL[d], m);
            if (!(fabs(x) < 1.0e6 * q.L[d])) set_status(a.status, GM_ERR_UNSUPPORTED);
            a.xw[3 * i + d] = w;
            a.mimg[3 * i + d] = m;
            c = (int)floor(w * q.inv_cs[d]);
            c = c < 0 ? 0 : (c >= q.nc[d] ? q.nc[d] - 1 : c);
            wf = (float)w;
        }
        const float w1 = __shfl_sync(full, wf, l1), w2 = __shfl_sync(full, wf, l2);
        const int c1 = __shfl_sync(full, c, l1), c2 = __shfl_sync(full, c, l2);
        if (act && d == 0) a.xs[i] = make_float4(wf, w1, w2, (float)(c + 3 * c1 + 9 * c2));
    }
}

// Accepted pairs of atom i (structure q) into the warp's buffer, in ascending j; returns the
// row length (entries beyond BR_CAP are counted, not stored)
__device__ int brute_row(const NlArgs &a, const NlStruct &q, int i, int lane, BrBuf &bb) {
    const unsigned full = 0xffffffffu, below = (1u << lane) - 1u;
    const float4 xi = a.xs[i];
    const float L0 = q.Lf[0], L1 = q.Lf[1], L2 = q.Lf[2];
    const float iL0 = 1.0f / L0, iL1 = 1.0f / L1, iL2 = 1.0f / L2;
    const float lo2 = a.rc2f - q.eps2, hi2 = a.rc2f + q.eps2;
    const float sc0 = (float)q.nc[0], sc1 = 3.0f * (float)q.nc[1], sc2 = 9.0f * (float)q.nc[2];
    const float soff = 13.0f - xi.w;
    int cnt = 0;
    // batches of BU chunks of 32 candidates: the tests of a batch are independent (one
    // vote for its band pairs), the ballots and stores follow in candidate order
    constexpr int BU = 8;
    const int aend = q.a0 + q.n;
    for (int b0 = q.a0; b0 < aend; b0 += 32 * BU) {
        float4 xb[BU];
#pragma unroll
        for (int u = 0; u < BU; ++u) {
            const int j = b0 + 32 * u + lane;
            xb[u] = j < aend ? a.xs[j] : make_float4(3.0e30f, 3.0e30f, 3.0e30f, 0.0f);
        }
        unsigned key[BU], inm = 0u, bandm = 0u;
#pragma unroll
        for (int u = 0; u < BU; ++u) {
            const int j = b0 + 32 * u + lane;
            // minimum image n = -rint(d / L) per axis (boxes of at least 2 r_cut: the one
            // image that can be within r_cut; atom i's own images cannot)
            const float f0 = xb[u].x - xi.x, f1 = xb[u].y - xi.y, f2 = xb[u].z - xi.z;
            const float n0 = -rintf(f0 * iL0), n1 = -rintf(f1 * iL1), n2 = -rintf(f2 * iL2);
            const float dx = fmaf(n0, L0, f0), dy = fmaf(n1, L1, f1), dz = fmaf(n2, L2, f2);
            const float r2 = dx * dx + dy * dy + dz * dz;
            const bool other = j < aend && j != i;
            inm |= (other && r2 < lo2) ? 1u << u : 0u;
            bandm |= (other && r2 >= lo2 && r2 <= hi2) ? 1u << u : 0u;  // band: exact FP64 test
            const float st = fmaf(n2, sc2, fmaf(n1, sc1, fmaf(n0, sc0, xb[u].w + soff)));
            const float img = fmaf(n2, 9.0f, fmaf(n1, 3.0f, n0 + 13.0f));
            // st 32 + img < 2^10 for a pair within r_cut, an integer: the low mantissa bits of
            // its sum with 2^23
            const unsigned v = (unsigned)__float_as_int(fmaf(st, 32.0f, img) + 8388608.0f);
            key[u] = (v << 22) | (unsigned)j;
        }
        if (__any_sync(full, bandm != 0u)) {
#pragma unroll
            for (int u = 0; u < BU; ++u) {
                if (!((bandm >> u) & 1u)) continue;
                const int j = b0 + 32 * u + lane;
                const float n0 = -rintf((xb[u].x - xi.x) * iL0), n1 = -rintf((xb[u].y - xi.y) * iL1),
                            n2 = -rintf((xb[u].z - xi.z) * iL2);
                if (exact_inside(a.xw, j, a.xw[3 * i], a.xw[3 * i + 1], a.xw[3 * i + 2], (int)n0, (int)n1, (int)n2,
                                 q, __dmul_rn(a.rc, a.rc)))
                    inm |= 1u << u;
            }
        }
#pragma unroll
        for (int u = 0; u < BU; ++u) {
            const bool in = (inm >> u) & 1u;
            const unsigned ball = __ballot_sync(full, in);
            const int pos = cnt + __popc(ball & below);
            if (in && pos < BR_CAP) bb.key[pos] = key[u];
            cnt += __popc(ball);
        }
    }
    return cnt;
}

// The same for a structure with some box edge shorter than 2 r_cut (but at least r_cut: one
// cell and images n in {-1, 0, 1} of the wrapped positions per axis, so the stencil index of
// the key stays below 27): per axis the minimum image and, when it is also within r_cut on
// that axis, the other neighbouring image; every combination is tested (at most 8 per
// candidate).  A lane's accepted entries of a chunk (0..8) are placed by a warp scan, in
// candidate order and, within a candidate, in image order, so that the counting sort of the
// emit orders the row by stencil cell, stable in j, as for the single-image boxes.
__device__ int brute_row_multi(const NlArgs &a, const NlStruct &q, int i, int lane, BrBuf &bb) {
    const unsigned full = 0xffffffffu;
    const float4 xi = a.xs[i];
    const float L0 = q.Lf[0], L1 = q.Lf[1], L2 = q.Lf[2];
    const float iL0 = 1.0f / L0, iL1 = 1.0f / L1, iL2 = 1.0f / L2;
    const float lo2 = a.rc2f - q.eps2, hi2 = a.rc2f + q.eps2;
    // an image farther than this from the centre on one axis is out of range (a margin above
    // the FP32 rounding of the per-axis displacement)
    const float axis_cut = sqrtf(hi2) * 1.0001f;
    const float sc0 = (float)q.nc[0], sc1 = 3.0f * (float)q.nc[1], sc2 = 9.0f * (float)q.nc[2];
    const float soff = 13.0f - xi.w;
    const int aend = q.a0 + q.n;
    int cnt = 0;
    const float4 far4 = make_float4(3.0e30f, 3.0e30f, 3.0e30f, 0.0f);
    float4 xn = q.a0 + lane < aend ? a.xs[q.a0 + lane] : far4;
    for (int b0 = q.a0; b0 < aend; b0 += 32) {
        const float4 xb = xn;
        const int j = b0 + lane;
        xn = b0 + 32 + lane < aend ? a.xs[b0 + 32 + lane] : far4;     // the next chunk in flight
        const float f0 = xb.x - xi.x, f1 = xb.y - xi.y, f2 = xb.z - xi.z;
        const float m0 = -rintf(f0 * iL0), m1 = -rintf(f1 * iL1), m2 = -rintf(f2 * iL2);
        const float e0 = fmaf(m0, L0, f0), e1 = fmaf(m1, L1, f1), e2 = fmaf(m2, L2, f2);
        // the other neighbouring image per axis, and whether it can be in range
        const float t0 = e0 > 0.0f ? -1.0f : 1.0f, t1 = e1 > 0.0f ? -1.0f : 1.0f, t2 = e2 > 0.0f ? -1.0f : 1.0f;
        const float g0 = fmaf(m0 + t0, L0, f0), g1 = fmaf(m1 + t1, L1, f1), g2 = fmaf(m2 + t2, L2, f2);
        const bool two0 = fabsf(g0) < axis_cut, two1 = fabsf(g1) < axis_cut, two2 = fabsf(g2) < axis_cut;
        const bool valid = j < aend;
        unsigned key[8], inm = 0u, bandm = 0u;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const bool x1 = k & 1, y1 = (k >> 1) & 1, z1 = (k >> 2) & 1;
            const bool act = valid && (!x1 || two0) && (!y1 || two1) && (!z1 || two2);
            const float dx = x1 ? g0 : e0, dy = y1 ? g1 : e1, dz = z1 ? g2 : e2;
            const float n0 = x1 ? m0 + t0 : m0, n1 = y1 ? m1 + t1 : m1, n2 = z1 ? m2 + t2 : m2;
            const float r2 = dx * dx + dy * dy + dz * dz;
            const bool other = act && (j != i || n0 != 0.0f || n1 != 0.0f || n2 != 0.0f);
            inm |= (other && r2 < lo2) ? 1u << k : 0u;
            bandm |= (other && r2 >= lo2 && r2 <= hi2) ? 1u << k : 0u;
            const float st = fmaf(n2, sc2, fmaf(n1, sc1, fmaf(n0, sc0, xb.w + soff)));
            const float img = fmaf(n2, 9.0f, fmaf(n1, 3.0f, n0 + 13.0f));
            const unsigned v = (unsigned)__float_as_int(fmaf(st, 32.0f, img) + 8388608.0f);
            key[k] = (v << 22) | (unsigned)j;
        }
        if (__any_sync(full, bandm != 0u)) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (!((bandm >> k) & 1u)) continue;
                const bool x1 = k & 1, y1 = (k >> 1) & 1, z1 = (k >> 2) & 1;
                const int n0 = (int)(x1 ? m0 + t0 : m0), n1 = (int)(y1 ? m1 + t1 : m1), n2 = (int)(z1 ? m2 + t2 : m2);
                if (exact_inside(a.xw, j, a.xw[3 * i], a.xw[3 * i + 1], a.xw[3 * i + 2], n0, n1, n2, q,
                                 __dmul_rn(a.rc, a.rc)))
                    inm |= 1u << k;
            }
        }
        const int c = __popc(inm);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(full, incl, o);
            if (lane >= o) incl += y;
        }
        int pos = cnt + incl - c;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if ((inm >> k) & 1u) {
                if (pos < BR_CAP) bb.key[pos] = key[k];
                ++pos;
            }
        }
        cnt += __shfl_sync(full, incl, 31);
    }
    return cnt;
}

// boxes shorter than 2 r_cut on some axis take the multi-image row
__device__ __forceinline__ bool brute_multi(const NlArgs &a, const NlStruct &q) {
    const float two = 2.001f * (float)a.rc;
    return q.Lf[0] < two || q.Lf[1] < two || q.Lf[2] < two;
}

__device__ __forceinline__ int brute_row_any(const NlArgs &a, const NlStruct &q, int i, int lane, BrBuf &bb) {
    return brute_multi(a, q) ? brute_row_multi(a, q, i, lane, bb) : brute_row(a, q, i, lane, bb);
}

// The buffered row (cnt <= BR_CAP entries) in stencil order, stable in j: into slab row i
// (codes; returns false when a shift has no code) or, with csr >= 0, into the CSR list at csr
// (slab rows go to dst: the slab row of i, or the warp buffer's row for the direct write)
__device__ bool brute_emit(const NlArgs &a, int i, int cnt, int lane, BrBuf &bb, int csr, unsigned *dst = nullptr) {
    const unsigned full = 0xffffffffu, below = (1u << lane) - 1u;
    if (lane < 32) bb.hist[lane] = 0;
    __syncwarp();
    for (int e = lane; e < cnt; e += 32) atomicAdd(&bb.hist[bb.key[e] >> 27], 1);
    __syncwarp();
    int h = lane < 27 ? bb.hist[lane] : 0, incl = h;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += y;
    }
    bb.run[lane] = incl - h;                                    // exclusive offsets per stencil cell
    __syncwarp();
    const int mi0 = a.mimg[3 * i], mi1 = a.mimg[3 * i + 1], mi2 = a.mimg[3 * i + 2];
    bool coded = true;
    for (int e0 = 0; e0 < cnt; e0 += 32) {
        const int e = e0 + lane;
        const bool v = e < cnt;
        const unsigned k = v ? bb.key[e] : 0u;
        const unsigned st = v ? k >> 27 : 31u;
        const unsigned m = __match_any_sync(full, st);
        const int pos = bb.run[st] + __popc(m & below);
        __syncwarp();
        if (v) {
            const int j = (int)(k & 0x3FFFFFu);
            const int img = (int)((k >> 22) & 31u);
            const int s0 = img % 3 - 1 - a.mimg[3 * j] + mi0;
            const int s1 = (img / 3) % 3 - 1 - a.mimg[3 * j + 1] + mi1;
            const int s2 = img / 9 - 1 - a.mimg[3 * j + 2] + mi2;
            if (csr >= 0) {
                store_pair(a, csr + pos, j, s0, s1, s2);
            } else {
                const unsigned code = shift_code(bytes3(s0, s1, s2));
                coded = coded && code != NL_NOCODE;
                (dst ? dst : a.slab + (size_t)i * a.maxn)[pos] = (unsigned)j | (code << 27);
            }
            if (lane == __ffs(m) - 1) bb.run[st] += __popc(m);
        }
        __syncwarp();
    }
    return __all_sync(full, coded);
}

// One atom per warp: rows into the slab (counts, redo marks as the cell-list search).  Row
// i = s nb + bid goes to warp (s + rot) mod NL_WARPS of block bid: rows spread over all
// blocks first, and the second half of the grid (the second block of each SM when the
// blocks fill the SMs in order) starts a quarter of the block further on, so that two
// blocks on one SM keep their busy warps on different schedulers.
//
// With at most one row per warp (N <= blocks x warps) the placed row stays in the warp's
// buffer (any length up to BR_CAP) and the compaction writes it into the CSR list from
// there (brute_direct); otherwise it goes to the slab.
__device__ __forceinline__ bool brute_direct(const NlArgs &a, int nb) { return a.N <= nb * NL_WARPS; }

__device__ void ph_search_brute(const NlArgs &a, int bid, int nb, const NlStruct *Ss, BrBuf *bufs,
                                const int32_t *sptr = nullptr) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    BrBuf &bb = bufs[warp];
    const bool direct = brute_direct(a, nb);
    if (lane == 0) bb.rowi = -1;
    auto row = [&](int i) {
        const NlStruct &q = Ss[sptr ? structure_in(sptr, a.B, i) : structure_of(a.atom_ptr, a.B, i)];
        const int cnt = brute_row_any(a, q, i, lane, bb);
        if (cnt > BR_CAP) {
            if (lane == 0) atomicExch(a.brute_over, 1);
            return;
        }
        bool over = !direct && cnt > a.maxn;
        if (!over) over = !brute_emit(a, i, cnt, lane, bb, -1, direct ? bb.row : nullptr);
        if (lane == 0) {
            a.counts[i] = cnt;
            a.redo[i] = over ? 1 : 0;
            if (over) nl_redo(a, i);
            if (direct && !over) {
                bb.rowi = i;
                bb.rowcnt = cnt;
            }
        }
    };
    const int rot = bid >= (nb >> 1) ? NL_WARPS / 4 : 0;
    for (int i = ((warp - rot + NL_WARPS) % NL_WARPS) * nb + bid; i < a.N; i += NL_WARPS * nb) row(i);
}

// Compaction after the slab pass: each warp copies NL_COPY_ROWS slab rows at a time into
// their CSR rows (all loads of a step before its stores); rows marked for a redo -- longer
// than the slab, or of structures that take the per-atom search -- are searched again
// straight into the CSR row.
constexpr int NL_COPY_ROWS = 4;

__device__ void ph_compact(const NlArgs &a, int bid, int nb, const int32_t *row_ptr, BrBuf *brute = nullptr) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned full = 0xffffffffu;
    if (__shfl_sync(full, lane == 0 ? (int)status_bad(a.status) : 0, 0)) return;
    const int gw = bid + nb * warp, nw = nb * NL_WARPS;
    if (brute && brute_direct(a, nb)) {                // the warp's own placed row, from its buffer
        const BrBuf &bb = brute[warp];
        const int i = bb.rowi;
        if (i >= 0) {
            const int r0 = row_ptr[i], cnt = bb.rowcnt;
            for (int k = lane; k < cnt; k += 32) {
                const unsigned e = bb.row[k], code = e >> 27;
                a.col[r0 + k] = (int)(e & 0x7FFFFFFu);
                a.shift[r0 + k] = make_char4((signed char)((int)(code % 3u) - 1), (signed char)((int)((code / 3u) % 3u) - 1),
                                             (signed char)((int)(code / 9u) - 1), 0);
            }
        }
    }
    for (int i0 = gw * NL_COPY_ROWS; !(brute && brute_direct(a, nb)) && i0 < a.N; i0 += nw * NL_COPY_ROWS) {
        int r0[NL_COPY_ROWS], cnt[NL_COPY_ROWS], kmax = 0;
#pragma unroll
        for (int u = 0; u < NL_COPY_ROWS; ++u) {
            const int i = i0 + u;
            r0[u] = 0;
            cnt[u] = 0;
            if (i < a.N) {
                r0[u] = row_ptr[i];
                cnt[u] = a.redo[i] ? 0 : row_ptr[i + 1] - r0[u];
            }
            kmax = max(kmax, cnt[u]);
        }
        for (int k0 = 0; k0 < kmax; k0 += 64) {
            unsigned e[NL_COPY_ROWS][2];
#pragma unroll
            for (int u = 0; u < NL_COPY_ROWS; ++u)
#pragma unroll
                for (int v = 0; v < 2; ++v) {
                    const int k = k0 + 32 * v + lane;
                    e[u][v] = k < cnt[u] ? a.slab[(size_t)(i0 + u) * a.maxn + k] : 0u;
                }
#pragma unroll
            for (int u = 0; u < NL_COPY_ROWS; ++u)
#pragma unroll
                for (int v = 0; v < 2; ++v) {
                    const int k = k0 + 32 * v + lane;
                    const unsigned code = e[u][v] >> 27;                 // 0..26 in rows that are copied
                    const int s0 = (int)(code % 3u) - 1, s1 = (int)((code / 3u) % 3u) - 1, s2 = (int)(code / 9u) - 1;
                    if (k < cnt[u]) {
                        a.col[r0[u] + k] = (int)(e[u][v] & 0x7FFFFFFu);
                        a.shift[r0[u] + k] = make_char4((signed char)s0, (signed char)s1, (signed char)s2, 0);
                    }
                }
        }
    }
    const int nredo = min(*a.n_redo, a.N);
    for (int r = gw; r < nredo; r += nw) {
        const int i = a.redo_list[r];
        if (brute) {                                   // rows of the brute-force search (<= BR_CAP)
            BrBuf &bb = brute[warp];
            const int cnt = brute_row_any(a, a.S[structure_of(a.atom_ptr, a.B, i)], i, lane, bb);
            brute_emit(a, i, min(cnt, BR_CAP), lane, bb, row_ptr[i]);
            continue;
        }
        const int c = a.cellid[i];
        const NlStruct &q = a.S[a.cstruct[c]];
        const float4 me = make_float4((float)a.xw[3 * i], (float)a.xw[3 * i + 1], (float)a.xw[3 * i + 2],
                                      __int_as_float(i));
        search_atom_generic<true>(a, q, c - q.cell0, me, lane, row_ptr[i]);
    }
}

// ------------------------------------------------------------------ kernels
enum NlPhase { PH_SETUP, PH_BIN, PH_SCAN_CELLS_ONE, PH_SCAN1_CELLS, PH_SCAN2_CELLS, PH_SCATTER, PH_SORT, PH_COUNT,
               PH_SCAN_ROWS_ONE, PH_SCAN1_ROWS, PH_SCAN2_ROWS, PH_FILL };
// with a slab, PH_COUNT is the single search pass and PH_FILL the compaction

__device__ __forceinline__ void run_phase(const NlArgs &a, int ph, int bid, int nb, float4 *smem) {
    switch (ph) {
    case PH_SETUP: ph_setup(a, bid, nb); break;
    case PH_BIN: ph_bin(a, bid, nb, a.S); break;
    case PH_SCAN_CELLS_ONE: ph_scan_one(a.ccount, a.cstart, *a.ncells, bid, 0, nullptr, a.status); break;
    case PH_SCAN1_CELLS: ph_scan1(a.ccount, a.cstart, *a.ncells, a.bsum, bid, nb); break;
    case PH_SCAN2_CELLS: ph_scan2(a.cstart, *a.ncells, a.bsum, bid, nb, 0, nullptr, a.status); break;
    case PH_SCATTER: ph_scatter(a, bid, nb, a.cstart); break;
    case PH_SORT: ph_sort(a, bid, nb); break;
    case PH_COUNT:
        if (a.block_items) {
            if (a.maxn > 0) ph_search_block<SM_SLAB>(a, bid, nb, smem);
            else ph_search_block<SM_COUNT>(a, bid, nb, smem);
        } else {
            if (a.maxn > 0) ph_search<SM_SLAB>(a, bid, nb, smem);
            else ph_search<SM_COUNT>(a, bid, nb, smem);
        }
        break;
    case PH_SCAN_ROWS_ONE: ph_scan_one(a.counts, a.row_ptr, a.N, bid, a.cap, a.n_pairs, a.status); break;
    case PH_SCAN1_ROWS: ph_scan1(a.counts, a.row_ptr, a.N, a.bsum, bid, nb); break;
    case PH_SCAN2_ROWS: ph_scan2(a.row_ptr, a.N, a.bsum, bid, nb, a.cap, a.n_pairs, a.status); break;
    default:
        if (a.maxn > 0) ph_compact(a, bid, nb, a.row_ptr);
        else if (a.block_items) ph_search_block<SM_FILL>(a, bid, nb, smem);
        else ph_search<SM_FILL>(a, bid, nb, smem);
        break;
    }
}

// All phases in one launch; the scans take one block when they are short (the decision is
// the same in every block: it reads the same counts).
// The brute-force search (grids already in Ss): true when it built the list (or gave up on
// an error), false when a row was longer than BR_CAP and the cell list must be built instead.
__device__ bool nl_brute_build(const NlArgs &a, int bid, int nb, NlStruct *Ss, int32_t *si, float4 *smem) {
    BrBuf *bufs = reinterpret_cast<BrBuf *>(reinterpret_cast<char *>(smem) + NL_BR_OFF);
    ph_wrap_brute(a, bid, nb, Ss);
    if (!nl_grid_sync(a.bar, a.status)) return true;
    ph_search_brute(a, bid, nb, Ss, bufs);
    if (!nl_grid_sync(a.bar, a.status)) return true;
    if (*reinterpret_cast<volatile int *>(a.brute_over) != 0) {
        if (bid == 0 && threadIdx.x == 0) *a.n_redo = 0;
        return false;
    }
    ph_scan_local(a.counts, a.N, si, bid, a.row_ptr, a.cap, a.n_pairs, a.status);
    if ((int64_t)si[a.N] > a.cap) return true;
    ph_compact(a, bid, nb, si, bufs);
    return true;
}

// The brute-force search for a batch of many small structures (the grids already in a.S, set
// up by block 0): wrap, search into the slab, the row scan over the whole batch, compaction.
// Returns false when a row was longer than BR_CAP (the cell-list phases build the list).
__device__ bool nl_brute_build_batch(const NlArgs &a, int bid, int nb, float4 *smem) {
    BrBuf *bufs = reinterpret_cast<BrBuf *>(reinterpret_cast<char *>(smem) + NL_BR_OFF);
    // each block copies the structure grids (up to 256) and atom_ptr into shared memory: the
    // structure of a row or an atom is then a search in shared memory, not eight dependent
    // global loads (256-box batch: build 188 -> 173 us)
    const NlStruct *Ss = a.S;
    if (a.B <= 256) {
        static_assert(sizeof(NlStruct) % 16 == 0, "16-byte copies of the structure grids");
        constexpr int W4 = (int)(sizeof(NlStruct) / 16);
        const float4 *src = reinterpret_cast<const float4 *>(a.S);
        float4 *dst = reinterpret_cast<float4 *>(smem);
        for (int k = threadIdx.x; k < a.B * W4; k += NL_THREADS) dst[k] = src[k];
        Ss = reinterpret_cast<const NlStruct *>(smem);
    }
    const int32_t *sptr = nullptr;
    if (a.B + 1 <= BR_PTR_MAX) {
        int32_t *sp = reinterpret_cast<int32_t *>(reinterpret_cast<char *>(smem) + NL_BR_PTR_OFF);
        for (int b = threadIdx.x; b <= a.B; b += NL_THREADS) sp[b] = a.atom_ptr[b];
        sptr = sp;
    }
    __syncthreads();
    ph_wrap_brute(a, bid, nb, Ss, sptr);
    if (!nl_grid_sync(a.bar, a.status)) return true;
    ph_search_brute(a, bid, nb, Ss, bufs, sptr);
    if (!nl_grid_sync(a.bar, a.status)) return true;
    if (*reinterpret_cast<volatile int *>(a.brute_over) != 0) {
        if (bid == 0 && threadIdx.x == 0) *a.n_redo = 0;
        return false;
    }
    if (a.N <= NL_SCAN_ONE_BLOCK) {
        run_phase(a, PH_SCAN_ROWS_ONE, bid, nb, smem);
    } else {
        run_phase(a, PH_SCAN1_ROWS, bid, nb, smem);
        if (!nl_grid_sync(a.bar, a.status)) return true;
        run_phase(a, PH_SCAN2_ROWS, bid, nb, smem);
    }
    if (!nl_grid_sync(a.bar, a.status)) return true;
    ph_compact(a, bid, nb, a.row_ptr, bufs);
    return true;
}

__global__ void __launch_bounds__(NL_THREADS, 2) k_nl_coop(NlArgs a) {
    extern __shared__ float4 nl_smem[];
    const int bid = blockIdx.x, nb = gridDim.x;
    if (nl_gated_off(a)) return;
    // failure-reporting tests: block 0 never arrives, so every other block's first (bounded)
    // grid barrier runs out and it returns with GM_ERR_TIMEOUT; the next build's memset
    // resets the barrier words
    if (a.debug_stall && bid == 0 && nb > 1) return;
    if (a.mid) {
        // every block sets up the grids; the brute-force search when the boxes allow it, else
        // (or after a row longer than BR_CAP) the phases below from the binning on -- the
        // setup published the grids, the cell count and the redo count as the setup phase does
        NlStruct *Ss = reinterpret_cast<NlStruct *>(nl_smem);
        ph_setup_local(a, bid, Ss);
        if (a.try_brute && nl_brute_eligible(a, Ss) &&
            nl_brute_build(a, bid, nb, Ss, reinterpret_cast<int32_t *>(nl_smem), nl_smem))
            return;
        for (int c = bid * NL_THREADS + threadIdx.x; c < a.ncmax; c += nb * NL_THREADS) a.cfill[c] = 0;
        if (!nl_grid_sync(a.bar, a.status)) return;
    }
    if (a.small) {
        // four barriers: every block sets up the grids and scans the short arrays itself
        NlStruct *Ss = reinterpret_cast<NlStruct *>(nl_smem);
        int32_t *si = reinterpret_cast<int32_t *>(nl_smem);
        ph_setup_local(a, bid, Ss);
        // a row longer than BR_CAP: the cell-list path below builds the list instead
        if (a.try_brute && nl_brute_eligible(a, Ss) && nl_brute_build(a, bid, nb, Ss, si, nl_smem)) return;
        for (int c = bid * NL_THREADS + threadIdx.x; c < a.ncmax; c += nb * NL_THREADS) a.cfill[c] = 0;
        ph_bin(a, bid, nb, Ss);
        if (!nl_grid_sync(a.bar, a.status)) return;
        const int ncells = *a.ncells;
        ph_scan_local(a.ccount, ncells, si, bid, a.cstart, 0, nullptr, a.status);
        ph_scatter(a, bid, nb, si);
        if (!nl_grid_sync(a.bar, a.status)) return;
        run_phase(a, PH_SORT, bid, nb, nl_smem);
        if (!nl_grid_sync(a.bar, a.status)) return;
        run_phase(a, PH_COUNT, bid, nb, nl_smem);
        if (!nl_grid_sync(a.bar, a.status)) return;
        ph_scan_local(a.counts, a.N, si, bid, a.row_ptr, a.cap, a.n_pairs, a.status);
        if ((int64_t)si[a.N] > a.cap) return;
        if (a.maxn > 0) {
            ph_compact(a, bid, nb, si);
        } else {
            if (!nl_grid_sync(a.bar, a.status)) return;        // the fill reads the published rows
            ph_search<SM_FILL>(a, bid, nb, nl_smem);
        }
        return;
    }
    if (!a.mid) {
        run_phase(a, PH_SETUP, bid, nb, nl_smem);
        if (!nl_grid_sync(a.bar, a.status)) return;
        // a batch of small structures: the brute-force search per structure (a row longer
        // than BR_CAP sends the build on to the phases below)
        if (a.try_brute && nl_brute_eligible(a, a.S) && nl_brute_build_batch(a, bid, nb, nl_smem)) return;
    }
    run_phase(a, PH_BIN, bid, nb, nl_smem);
    if (!nl_grid_sync(a.bar, a.status)) return;
    if (*a.ncells <= NL_SCAN_ONE_BLOCK) {
        run_phase(a, PH_SCAN_CELLS_ONE, bid, nb, nl_smem);
    } else {
        run_phase(a, PH_SCAN1_CELLS, bid, nb, nl_smem);
        if (!nl_grid_sync(a.bar, a.status)) return;
        run_phase(a, PH_SCAN2_CELLS, bid, nb, nl_smem);
    }
    if (!nl_grid_sync(a.bar, a.status)) return;
    run_phase(a, PH_SCATTER, bid, nb, nl_smem);
    if (!nl_grid_sync(a.bar, a.status)) return;
    run_phase(a, PH_SORT, bid, nb, nl_smem);
    if (!nl_grid_sync(a.bar, a.status)) return;
    run_phase(a, PH_COUNT, bid, nb, nl_smem);
    if (!nl_grid_sync(a.bar, a.status)) return;
    if (a.N <= NL_SCAN_ONE_BLOCK) {
        run_phase(a, PH_SCAN_ROWS_ONE, bid, nb, nl_smem);
    } else {
        run_phase(a, PH_SCAN1_ROWS, bid, nb, nl_smem);
        if (!nl_grid_sync(a.bar, a.status)) return;
        run_phase(a, PH_SCAN2_ROWS, bid, nb, nl_smem);
    }
    if (!nl_grid_sync(a.bar, a.status)) return;
    run_phase(a, PH_FILL, bid, nb, nl_smem);
}

// zero p[0..n) when *gate != 0 (the cleared words of a gated build)
__global__ void __launch_bounds__(256) k_nl_zero_gated(int32_t *p, int n, const int32_t *gate) {
    griddep_wait();
    if (*reinterpret_cast<const volatile int32_t *>(gate) == 0) return;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) p[q] = 0;
}

__global__ void __launch_bounds__(NL_THREADS, 2) k_nl_phase(NlArgs a, int ph) {
    extern __shared__ float4 nl_smem[];
    if (nl_gated_off(a)) return;
    run_phase(a, ph, blockIdx.x, gridDim.x, nl_smem);
}

// ------------------------------------------------------------------ host
struct NlWs {
    NlStruct *S;
    int32_t *ncells, *mimg, *cellid, *ccount, *cstart, *cfill, *unsorted, *counts, *bsum, *redo_list, *n_redo;
    int32_t *cstruct, *item_ctr, *brute_over;
    uint32_t *xsm, *mpk;
    uint8_t *redo;
    uint32_t *slab;
    unsigned *bar;
    double *xw;
    float4 *xs;
};

static NlWs carve_nl(Carve &c, int B, int N) {
    NlWs w;
    const int ncmax = N + B;
    const size_t n1 = N > 0 ? (size_t)N : 1;
    w.S = c.take<NlStruct>(B);
    w.ncells = c.take<int32_t>(1);

    w.xw = c.take<double>(3 * n1);
    w.mimg = c.take<int32_t>(3 * n1);
    w.cellid = c.take<int32_t>(n1);
    w.ccount = c.take<int32_t>(ncmax + 64);                        // histogram, then the barrier words
    w.bar = reinterpret_cast<unsigned *>(w.ccount + ncmax + 32);
    w.item_ctr = w.ccount + ncmax + 40;                            // search item counters (same memset)
    w.brute_over = w.ccount + ncmax + 44;                          // brute-force overflow flag (same memset)
    w.cstruct = c.take<int32_t>(ncmax);
    w.cstart = c.take<int32_t>(ncmax + 1);
    w.cfill = c.take<int32_t>(ncmax);
    w.unsorted = c.take<int32_t>(n1);
    w.xs = c.take<float4>(n1);
    w.xsm = c.take<uint32_t>(n1);
    w.mpk = c.take<uint32_t>(n1);
    w.redo = c.take<uint8_t>(n1);
    w.redo_list = c.take<int32_t>(n1);
    w.n_redo = c.take<int32_t>(1);
    w.counts = c.take<int32_t>(n1);
    w.bsum = c.take<int32_t>(NL_MAX_BLOCKS);
    return w;
}

// Slab row length for a list of `capacity` pairs: 1.25x the mean row plus a margin, in
// multiples of 32 (rows longer than this are searched again during the compaction).
static int nl_slab_row(int64_t capacity, int n_atoms) {
    if (n_atoms <= 0 || n_atoms >= (1 << 27) || capacity <= 0) return 0;
    int64_t m = (capacity * 5) / (4 * (int64_t)n_atoms) + 16;
    m = (m + 31) / 32 * 32;
    return (int)(m < 64 ? 64 : (m > 4096 ? 4096 : m));
}

size_t nl_workspace_min_bytes(int n_struct, int n_atoms) {
    Carve c(reinterpret_cast<void *>(256), ~size_t(0) >> 1);
    carve_nl(c, n_struct, n_atoms);
    return c.off + 256;
}

size_t nl_workspace_bytes(int n_struct, int n_atoms, int64_t capacity) {
    const int maxn = nl_slab_row(capacity, n_atoms);
    return nl_workspace_min_bytes(n_struct, n_atoms) + (maxn > 0 ? (size_t)n_atoms * maxn * sizeof(uint32_t) + 256 : 0);
}

struct NlDevice {
    bool init = false;
    int sms = 0, coop_blocks = 0;
};

static NlDevice &nl_device() {
    static NlDevice d[64];
    int dev = 0;
    cudaGetDevice(&dev);
    NlDevice &x = d[dev & 63];
    if (!x.init) {
        cudaDeviceGetAttribute(&x.sms, cudaDevAttrMultiProcessorCount, dev);
        int coop = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        cudaFuncSetAttribute(k_nl_coop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NL_SMEM);
        cudaFuncSetAttribute(k_nl_phase, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NL_SMEM);
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_nl_coop, NL_THREADS, NL_SMEM) != cudaSuccess)
            per_sm = 0;
        x.coop_blocks = coop ? per_sm * x.sms : 0;
        x.init = true;
    }
    return x;
}

// parts per home cell: enough work items for the warps of a small system, few repeated
// candidate reads for a large one
static int nl_auto_split(int N, bool block_items) {
    if (block_items) return N < 4096 ? 2 : 1;
    return N < 65536 ? 2 : 1;
}

gm_status nl_build(const gm_system &sys, double r_cut, int n_species, gm_nlist &nl, void *ws, size_t ws_bytes,
                   int32_t *status, cudaStream_t st, const NlTuning &tune, const int32_t *gate) {
    const int B = sys.n_structures, N = sys.n_atoms;
    Carve c(ws, ws_bytes);
    NlWs w = carve_nl(c, B, N);
    if (!c.ok) return GM_ERR_WORKSPACE;
    // the single-pass search when the workspace also holds the slab, else the two-pass one
    int maxn = tune.two_pass ? 0 : nl_slab_row(nl.capacity, N);
    w.slab = nullptr;
    if (maxn > 0) {
        w.slab = c.take<uint32_t>((size_t)N * maxn);
        if (!c.ok) { maxn = 0; w.slab = nullptr; }
    }
    NlArgs a;
    a.N = N;
    a.B = B;
    a.n_species = n_species;
    a.ncmax = N + B;
    // block items for small systems and for batches of small boxes (few cells per structure)
    a.block_items = tune.items == 1 ? 1 : (tune.items == 2 ? 0 : ((N < 16384 || N < 2048 * B) ? 1 : 0));
    a.split = tune.split > 0 ? tune.split : nl_auto_split(N, a.block_items != 0);
    a.atom_ptr = sys.atom_ptr;
    a.pos = sys.pos;
    a.species = sys.species;
    a.cell = sys.cell;
    a.pbc = sys.pbc;
    a.rc = r_cut;
    a.rc2f = (float)(r_cut * r_cut);
    a.S = w.S;
    a.ncells = w.ncells;
    a.cellid = w.cellid;
    a.cstruct = w.cstruct;
    a.item_ctr = w.item_ctr;
    a.ccount = w.ccount;
    a.cstart = w.cstart;
    a.cfill = w.cfill;
    a.unsorted = w.unsorted;
    a.counts = w.counts;
    a.bsum = w.bsum;
    a.mimg = w.mimg;
    a.xw = w.xw;
    a.xs = w.xs;
    a.xsm = w.xsm;
    a.mpk = w.mpk;
    a.slab = w.slab;
    a.maxn = maxn;
    a.redo = w.redo;
    a.redo_list = w.redo_list;
    a.n_redo = w.n_redo;
    a.row_ptr = nl.row_ptr;
    a.col = nl.col;
    a.shift = reinterpret_cast<char4 *>(nl.shift);
    a.cap = nl.capacity;
    a.n_pairs = nl.n_pairs;
    a.bar = w.bar;
    a.status = status;
    a.gate = gate;
    a.debug_stall = tune.debug_stall;

    NlDevice &dev = nl_device();
    const int ncmax = N + B;
    // cell histogram and barrier words start at zero (a gated build clears them only when it
    // will run: a kernel that reads the gate, in place of the memset)
    if (gate) {
        const int n0 = ncmax + 64;
        launch_pdl(k_nl_zero_gated, dim3((n0 + 1023) / 1024), dim3(256), 0, st, w.ccount, n0, gate);
        note_launches(1);
    } else if (cudaMemsetAsync(w.ccount, 0, sizeof(int32_t) * ((size_t)ncmax + 64), st) != cudaSuccess) {
        return GM_ERR_CUDA;
    }
    a.small = (N + B <= NL_SCAN_ONE_BLOCK && B <= 256) ? 1 : 0;
    // brute-force search (small systems and batches of small structures whose boxes are at least
    // r_cut long; decided on the device) unless the work items are set to cells, or there is no
    // slab
    a.try_brute = (tune.items == 0 || tune.items == 3) && a.maxn > 0 ? 1 : 0;
    a.mid = (!a.small && a.try_brute && N + B <= 2 * NL_SCAN_ONE_BLOCK && B <= 256) ? 1 : 0;
    a.brute_over = w.brute_over;
    auto clampi = [](long long v, long long lo, long long hi) { return (int)(v < lo ? lo : (v > hi ? hi : v)); };
    if (tune.mode != GM_NL_MODE_PHASES && dev.coop_blocks > 0) {
        // one cooperative launch, at most as many blocks as are co-resident
        const long long want = tune.blocks > 0 ? tune.blocks : 2LL * dev.sms;
        const int grid = clampi(want, 1, dev.coop_blocks < NL_MAX_BLOCKS ? dev.coop_blocks : NL_MAX_BLOCKS);
        StageScope sc(ST_NL_COOP, st);

        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(NL_THREADS);
        cfg.dynamicSmemBytes = NL_SMEM;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cudaLaunchKernelEx(&cfg, k_nl_coop, a) != cudaSuccess) return GM_ERR_CUDA;
        note_launches(1);
        return cudaPeekAtLastError() == cudaSuccess ? GM_OK : GM_ERR_CUDA;
    }
    // one launch per phase
    const int g_setup = clampi((ncmax + NL_THREADS - 1) / NL_THREADS, 1, NL_MAX_BLOCKS);
    const int g_atoms = clampi((N + NL_THREADS - 1) / NL_THREADS, 1, NL_MAX_BLOCKS);
    const int g_cells_scan = clampi((ncmax + NL_SCAN_SUB - 1) / NL_SCAN_SUB, 1, NL_MAX_BLOCKS);
    const int g_rows_scan = clampi((N + NL_SCAN_SUB - 1) / NL_SCAN_SUB, 1, NL_MAX_BLOCKS);
    const int g_sort = clampi((ncmax + NL_WARPS - 1) / NL_WARPS, 1, NL_MAX_BLOCKS);
    const int g_search =
        clampi(tune.blocks > 0 ? tune.blocks
                               : (a.block_items ? (long long)ncmax * a.split
                                                : ((long long)ncmax * a.split + NL_WARPS - 1) / NL_WARPS),
               1, 8LL * dev.sms);
    std::optional<StageScope> scope;
    int launches = 0;
    auto phase = [&](int grid, int ph) {
        const bool search = ph == PH_COUNT || (ph == PH_FILL && maxn == 0);
        k_nl_phase<<<grid, NL_THREADS, search ? NL_SMEM : 0, st>>>(a, ph);
        ++launches;
    };
    scope.emplace(ST_NL_BIN, st);
    phase(g_setup, PH_SETUP);
    phase(g_atoms, PH_BIN);
    if (ncmax <= NL_SCAN_ONE_BLOCK) {
        phase(1, PH_SCAN_CELLS_ONE);
    } else {
        phase(g_cells_scan, PH_SCAN1_CELLS);
        phase(g_cells_scan, PH_SCAN2_CELLS);
    }
    phase(g_atoms, PH_SCATTER);
    phase(g_sort, PH_SORT);
    scope.reset();
    scope.emplace(ST_NL_COUNT, st);
    phase(g_search, PH_COUNT);
    scope.reset();
    scope.emplace(ST_NL_SCAN, st);
    if (N <= NL_SCAN_ONE_BLOCK) {
        phase(1, PH_SCAN_ROWS_ONE);
    } else {
        phase(g_rows_scan, PH_SCAN1_ROWS);
        phase(g_rows_scan, PH_SCAN2_ROWS);
    }
    scope.reset();
    scope.emplace(ST_NL_FILL, st);
    phase(maxn > 0 ? clampi(((long long)N + NL_WARPS * NL_COPY_ROWS - 1) / (NL_WARPS * NL_COPY_ROWS), 1, 8LL * dev.sms)
                   : g_search,
          PH_FILL);
    note_launches(launches);
    scope.reset();
    return cudaPeekAtLastError() == cudaSuccess ? GM_OK : GM_ERR_CUDA;
}

}  // namespace gm
