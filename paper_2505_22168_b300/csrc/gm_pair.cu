// gm_pair.cu -- per-pair kernels: Gaussian moments (Eq. basis_fn) and forces.
//
// One group of TPA lanes per centre atom i walks i's CSR row; lanes take every TPA-th
// neighbour, so a warp covers 32/TPA atoms.  Per pair: the minimum-image displacement
// d = (r_j - r_i) + n.L is formed to FP64 accuracy (error-free FP32 transforms of hi/lo
// position splits, see disp_axis) and rounded to FP32; everything after that (r, rhat,
// basis, radial functions, monomials) is FP32.
//
// Moments:  Psi_i[s][c] = sum_j R_s(r_ij) m_c(rhat_ij)  (unique components m_c, see
//           gm_common.cuh), reduced across the TPA lanes with warp shuffles.
// Forces:   given g_i[s][c] = dE/dPsi_i[s][c], the pair gradient is
//              dE/dd_b = u_b (sum_c A'_c m_c - (1/r) sum_c L_c A_c m_c) + (1/r) sum_c A_c dm_c/du_b
//           with A_c = sum_s g[s][c] R_s and A'_c = sum_s g[s][c] R'_s (using Euler's
//           relation sum_a u_a dm_c/du_a = L_c m_c for the tangential projection).
//           F_i += dE/dd_ij and F_j -= dE/dd_ij (float atomics for the j side), and the
//           per-atom virial -d (x) dE/dd is accumulated for an FP64 per-structure sum.
#include "gm_internal.h"
#include "gm_pair.h"

namespace gm {

__device__ __forceinline__ int clamp_species(int z, int S, int32_t *status) {
    if (z < 0 || z >= S) {
        set_status(status, GM_ERR_SPECIES);
        return z < 0 ? 0 : S - 1;
    }
    return z;
}

// One axis of d = (x_j - x_i) + s L from hi/lo FP32 splits of the FP64 operands
// (x = x_h + x_l, L = L_h + L_l): the large terms are combined with error-free transforms
// (TwoSum of the hi difference, TwoProduct of s L_h, TwoSum of the two), the small terms are
// added in FP32, and the sum is rounded once.  The result is the FP32 rounding of the FP64
// displacement to within one ulp (rounded twice there), at FP32 cost: B300 issues FP64
// arithmetic at a small fraction of the FP32 rate.
__device__ __forceinline__ float disp_axis(float xjh, float xjl, float xih, float xil, float s, float Lh, float Ll) {
    const float h1 = xjh - xih;                       // TwoSum(xjh, -xih)
    const float b1 = h1 - xjh;
    const float l1 = (xjh - (h1 - b1)) + (-xih - b1);
    const float h2 = s * Lh;                          // TwoProduct(s, Lh)
    const float l2 = fmaf(s, Lh, -h2);
    const float h3 = h1 + h2;                         // TwoSum(h1, h2)
    const float b3 = h3 - h1;
    const float l3 = (h1 - (h3 - b3)) + (h2 - b3);
    const float lo = ((l1 + l2) + l3) + ((xjl - xil) + s * Ll);
    return h3 + lo;
}

// |d| and 1/|d| of a pair from one hardware reciprocal square root (relative error a few
// 2^-24 each, against the correctly rounded square root and division it replaces; d is never
// zero for a listed pair)
__device__ __forceinline__ void pair_length(float fx, float fy, float fz, float &r, float &rinv) {
    const float r2 = fx * fx + fy * fy + fz * fz;
    rinv = rsqrtf(r2);
    r = r2 * rinv;
}

// One neighbour of a row: index, shift, hi/lo position (species in ph.w) and, for the
// tangent kernels, its velocity (the direction the positions move along).
struct NextPair {
    int j;
    bool ok;
    char4 sh;
    float4 ph, pl;
    float vx, vy, vz;
};

// Gather pipeline over the pairs p0, p0 + step, ... < p1 of a row, U pairs per call: while
// pairs i .. i+U-1 are computed, the positions of the next U pairs and the indices of the U
// after those are in flight, so the dependent index -> position gather costs no latency
// inside the loop.
template <int U>
struct PairPipe {
    const float *vel;         // per-atom velocities [N][3] gathered with the positions (or null)
    int p1, step, q;          // q: first pair whose index is loaded next
    int jn[U];                // indices, shifts and flags two groups ahead
    char4 shn[U];
    bool okn[U];
    NextPair nx[U];           // the next group (position loads issued)
    __device__ __forceinline__ void index(const PairArgs &a, int p, int &j, char4 &sh, bool &ok) const {
        ok = false;
        if (p < p1) {
            j = a.col[p];
            sh = a.shift[p];
            ok = (unsigned)j < (unsigned)a.N;
            if (!ok) set_status(a.status, GM_ERR_ARG);
        }
    }
    __device__ __forceinline__ void gather(const PairArgs &a) {
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (nx[u].ok) {
                nx[u].ph = a.pos_hi[nx[u].j];
                nx[u].pl = a.pos_lo[nx[u].j];
                if (vel) {
                    nx[u].vx = vel[3 * nx[u].j];
                    nx[u].vy = vel[3 * nx[u].j + 1];
                    nx[u].vz = vel[3 * nx[u].j + 2];
                }
            }
    }
    __device__ __forceinline__ PairPipe(const PairArgs &a, int p0, int p1_, int step_, const float *vel_ = nullptr)
        : vel(vel_), p1(p1_), step(step_) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            index(a, p0 + u * step, nx[u].j, nx[u].sh, nx[u].ok);
            index(a, p0 + (U + u) * step, jn[u], shn[u], okn[u]);
        }
        gather(a);
        q = p0 + 2 * U * step;
    }
    // the current group; the pipeline advances by U pairs
    __device__ __forceinline__ void next(const PairArgs &a, NextPair (&cur)[U]) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            cur[u] = nx[u];
            nx[u].j = jn[u];
            nx[u].sh = shn[u];
            nx[u].ok = okn[u];
        }
        gather(a);
#pragma unroll
        for (int u = 0; u < U; ++u) index(a, q + u * step, jn[u], shn[u], okn[u]);
        q += U * step;
    }
    __device__ __forceinline__ NextPair next(const PairArgs &a) {
        NextPair cur[U];
        next(a, cur);
        return cur[0];
    }
};

// The centre atom's position and its box edges as hi/lo FP32 pairs.
struct Centre {
    float4 ph, pl;
    float Lh[3], Ll[3];
    __device__ __forceinline__ Centre(const PairArgs &a, int atom, int b) {
        ph = a.pos_hi[atom];
        pl = a.pos_lo[atom];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double L = a.cell[9 * b + 4 * d];
            Lh[d] = (float)L;
            Ll[d] = (float)(L - (double)Lh[d]);
        }
    }
    __device__ __forceinline__ void displacement(const NextPair &c, float &fx, float &fy, float &fz) const {
        fx = disp_axis(c.ph.x, c.pl.x, ph.x, pl.x, (float)c.sh.x, Lh[0], Ll[0]);
        fy = disp_axis(c.ph.y, c.pl.y, ph.y, pl.y, (float)c.sh.y, Lh[1], Ll[1]);
        fz = disp_axis(c.ph.z, c.pl.z, ph.z, pl.z, (float)c.sh.z, Lh[2], Ll[2]);
    }
};

// hi/lo FP32 split of the FP64 positions (once per atom), the species index carried in the
// hi word's w lane (so the neighbour gather brings it along); also clears the force array
// the force kernel accumulates into, when given
__global__ void __launch_bounds__(256) k_split_pos(int N, const double *__restrict__ pos,
                                                   const int32_t *__restrict__ species, float4 *__restrict__ hi,
                                                   float4 *__restrict__ lo, float *__restrict__ zero_F,
                                                   unsigned long long *__restrict__ zero_acc, int n_acc) {
    griddep_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (zero_acc)
        for (int q = i; q < n_acc; q += gridDim.x * blockDim.x) zero_acc[q] = 0ull;
    if (i >= N) return;
    if (zero_F) {
        zero_F[3 * i] = 0.0f;
        zero_F[3 * i + 1] = 0.0f;
        zero_F[3 * i + 2] = 0.0f;
    }
    float h[3], l[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double x = pos[3 * i + d];
        h[d] = (float)x;
        l[d] = (float)(x - (double)h[d]);
    }
    hi[i] = make_float4(h[0], h[1], h[2], __int_as_float(species[i]));
    lo[i] = make_float4(l[0], l[1], l[2], 0.0f);
}

void launch_split_pos(int N, const double *pos, const int32_t *species, float4 *hi, float4 *lo, float *zero_F,
                      unsigned long long *zero_acc, int n_acc, cudaStream_t st) {
    if (N <= 0) return;
    launch_pdl(k_split_pos, dim3((N + 255) / 256), dim3(256), 0, st, N, pos, species, hi, lo, zero_F, zero_acc, n_acc);
    note_launches(1);
}

// Block shape of the moments kernel: with 8 or more lanes per atom (small systems) 128-thread
// blocks at up to 170 registers, so that three blocks (12 warps) share an SM and a 1536-atom
// system runs in one wave; with fewer lanes 256-thread blocks and two pairs per iteration.
template <int TPA> __host__ __device__ constexpr int moments_threads() { return TPA >= 8 ? 128 : 256; }
template <int TPA, int BAS>
__global__ void __launch_bounds__(moments_threads<TPA>(), TPA >= 8 ? 3 : 1) k_moments(PairArgs a,
                                                                                   float *__restrict__ psi) {
    extern __shared__ __align__(16) float sbeta[];
    stage_beta(a.beta, a.S, sbeta);
    griddep_wait();
    __syncthreads();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int atom = g / TPA, sub = g % TPA;
    const bool active = atom < a.N && !status_bad(a.status);
    float acc[NPSI];
#pragma unroll
    for (int q = 0; q < NPSI; ++q) acc[q] = 0.0f;
    if (active) {
        const int b = structure_of(a.atom_ptr, a.B, atom);
        const Centre ce(a, atom, b);
        const int zsi = clamp_species(a.species[atom], a.S, a.status);
        const float *brow = sbeta + zsi * a.S * (NR * BETA_ROW);
        const int p1 = a.row_ptr[atom + 1];
        // U pairs per iteration (independent work for the latency-bound pair math); a missing
        // second pair contributes exact zeros, so the sums are those of one pair at a time in
        // row order
        constexpr int U = TPA >= 8 ? 1 : 2;
        PairPipe<U> pp(a, a.row_ptr[atom] + sub, p1, TPA);
        for (int p = a.row_ptr[atom] + sub; p < p1; p += U * TPA) {
            NextPair cur[U];
            pp.next(a, cur);
            float R[U][NR], m[U][NC];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                float fx = 1.0f, fy = 0.0f, fz = 0.0f;
                int zj = 0;
                if (cur[u].ok) {
                    ce.displacement(cur[u], fx, fy, fz);
                    zj = clamp_species(__float_as_int(cur[u].ph.w), a.S, a.status);
                }
                float r, rinv;
                pair_length(fx, fy, fz, r, rinv);
                float B[NB], dB[NB];
                radial_basis<false, BAS>(a.rc, r, B, dB);
                const float w = cur[u].ok ? 1.0f : 0.0f;
                float Rp[NR];
                radial_combine<false>(brow + zj * (NR * BETA_ROW), B, dB, R[u], Rp);
#pragma unroll
                for (int s = 0; s < NR; ++s) R[u][s] *= w;
                monomials(fx * rinv, fy * rinv, fz * rinv, m[u]);
            }
#pragma unroll
            for (int s = 0; s < NR; ++s)
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    float t = acc[s * NC + c];
#pragma unroll
                    for (int u = 0; u < U; ++u) t = fmaf(R[u][s], m[u][c], t);
                    acc[s * NC + c] = t;
                }
        }
    }
    if (TPA >= 8) {
        // reduce-scatter by recursive halving: after log2(TPA) steps each lane holds
        // 128/TPA consecutive sums (of 100 values padded to 128), ~124 shuffles for TPA 32
        float v[128];
#pragma unroll
        for (int q = 0; q < 128; ++q) v[q] = q < NPSI ? acc[q] : 0.0f;
        int start = 0;
#pragma unroll
        for (int off = TPA / 2, len = 64; off > 0; off >>= 1, len >>= 1) {
            const bool upper = (sub & off) != 0;
#pragma unroll
            for (int q = 0; q < len; ++q) {
                const float send = upper ? v[q] : v[len + q];
                const float keep = upper ? v[len + q] : v[q];
                v[q] = keep + __shfl_xor_sync(0xffffffffu, send, off);
            }
            start += upper ? len : 0;
        }
        if (!active) return;
        float *out = psi + (size_t)atom * NPSI;
        constexpr int per = 128 / TPA;
#pragma unroll
        for (int q = 0; q < per; ++q)
            if (start + q < NPSI) out[start + q] = v[q];
        return;
    }
    if (TPA > 1) {
#pragma unroll
        for (int off = TPA / 2; off > 0; off >>= 1)
#pragma unroll
            for (int q = 0; q < NPSI; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
    }
    if (!active) return;
    float *out = psi + (size_t)atom * NPSI;
    if (TPA == 1) {
        float4 *o4 = reinterpret_cast<float4 *>(out);
#pragma unroll
        for (int q = 0; q < NPSI / 4; ++q) o4[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    } else {
#pragma unroll
        for (int q = 0; q < NPSI; ++q)
            if (q % TPA == sub) out[q] = acc[q];
    }
}

// Moments with the components split over a lane pair (large systems, TPA = 2 or 4 lanes per
// atom).  The TPA lanes of an atom form TPA/2 groups of two; the two lanes of a group (role
// h = lane & 1) take one pair each per step, evaluate its radial part once, and swap their
// R_s and the half of the monomials the other lane keeps: lane h accumulates the components
// c in [10h, 10h + 10) of both pairs, 50 sums instead of 100, which halves the registers of
// the one-lane kernel (two blocks per SM instead of one) without repeating the radial part.
// With TPA = 4 the two groups take alternate pair couples of the row and add their sums with
// one shuffle at the end.
constexpr int NCH = NC / 2;
template <int TPA, int BAS>
__global__ void __launch_bounds__(256, 2) k_moments_cs(PairArgs a, float *__restrict__ psi) {
    static_assert(TPA == 2 || TPA == 4, "component-split moments take 2 or 4 lanes per atom");
    extern __shared__ __align__(16) float sbeta[];
    stage_beta(a.beta, a.S, sbeta);
    griddep_wait();
    __syncthreads();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int atom = g / TPA, sub = g % TPA, h = sub & 1, grp = sub >> 1;
    const bool active = atom < a.N && !status_bad(a.status);
    // the two lanes of this group (they run the same steps of the same row)
    const unsigned pmask = 3u << ((threadIdx.x & 31) & ~1);
    float acc[NR][NCH];
#pragma unroll
    for (int s = 0; s < NR; ++s)
#pragma unroll
        for (int k = 0; k < NCH; ++k) acc[s][k] = 0.0f;
    if (active) {
        const int b = structure_of(a.atom_ptr, a.B, atom);
        const Centre ce(a, atom, b);
        const int zsi = clamp_species(a.species[atom], a.S, a.status);
        const float *brow = sbeta + zsi * a.S * (NR * BETA_ROW);
        const int p0 = a.row_ptr[atom], p1 = a.row_ptr[atom + 1];
        // this lane's pairs: p0 + 2 grp + h, then every TPA-th
        PairPipe<1> pp(a, p0 + 2 * grp + h, p1, TPA);
        for (int p = p0 + 2 * grp; p < p1; p += TPA) {
            const NextPair cur = pp.next(a);
            float fx = 1.0f, fy = 0.0f, fz = 0.0f;
            int zj = 0;
            if (cur.ok) {
                ce.displacement(cur, fx, fy, fz);
                zj = clamp_species(__float_as_int(cur.ph.w), a.S, a.status);
            }
            float r, rinv;
            pair_length(fx, fy, fz, r, rinv);
            float B[NB], dB[NB];
            radial_basis<false, BAS>(a.rc, r, B, dB);
            float R[NR], Rp[NR];
            radial_combine<false>(brow + zj * (NR * BETA_ROW), B, dB, R, Rp);
            const float w = cur.ok ? 1.0f : 0.0f;    // a missing second pair adds exact zeros
#pragma unroll
            for (int s = 0; s < NR; ++s) R[s] *= w;
            float m[NC];
            monomials(fx * rinv, fy * rinv, fz * rinv, m);
            // keep one half of this pair's monomials, send the other half and R to the partner
            float mk[NCH], mo[NCH], Ro[NR];
#pragma unroll
            for (int k = 0; k < NCH; ++k) {
                mk[k] = h ? m[NCH + k] : m[k];
                mo[k] = __shfl_xor_sync(pmask, h ? m[k] : m[NCH + k], 1);
            }
#pragma unroll
            for (int s = 0; s < NR; ++s) Ro[s] = __shfl_xor_sync(pmask, R[s], 1);
#pragma unroll
            for (int s = 0; s < NR; ++s)
#pragma unroll
                for (int k = 0; k < NCH; ++k) acc[s][k] = fmaf(Ro[s], mo[k], fmaf(R[s], mk[k], acc[s][k]));
        }
    }
    if (TPA == 4) {
#pragma unroll
        for (int s = 0; s < NR; ++s)
#pragma unroll
            for (int k = 0; k < NCH; ++k) acc[s][k] += __shfl_xor_sync(0xffffffffu, acc[s][k], 2);
    }
    if (!active) return;
    // lane h holds Psi[s][10h + k]; with TPA = 4 the two groups store alternate radial functions
    float2 *out = reinterpret_cast<float2 *>(psi + (size_t)atom * NPSI);
#pragma unroll
    for (int s = 0; s < NR; ++s) {
        if (TPA == 4 && (s & 1) != grp) continue;
#pragma unroll
        for (int k = 0; k < NCH / 2; ++k)
            out[(s * NC + h * NCH) / 2 + k] = make_float2(acc[s][2 * k], acc[s][2 * k + 1]);
    }
}

// Block shape and gradient storage of the force kernel.  With 4 or more lanes per atom the
// atom's dE/dPsi (identical for its lanes) sits once in shared memory, transposed to
// [component][radial function] rows of 8 (one 16-byte and one 4-byte broadcast load per
// component; atoms 164 floats apart, so the up to 8 atoms of a warp hit distinct banks), and
// 128-thread blocks run four per SM; with fewer lanes each lane keeps it in registers.
template <int TPA> __host__ __device__ constexpr bool forces_gsmem() { return TPA >= 4; }
template <int TPA> __host__ __device__ constexpr int forces_threads() { return TPA >= 4 ? 128 : 256; }
constexpr int FG_ROW = 164;
static_assert(FG_ROW >= NC * 8 && FG_ROW % 4 == 0 && FG_ROW % 32 == 4, "dE/dPsi rows: 16-byte aligned, distinct banks");
// VIR: the per-atom virial is accumulated and stored (vir_atom), else not formed at all.
// heads > 1 (shallow-ensemble heads, no virial): heads x N virtual atoms, virtual atom
// h N + i taking dE/dPsi row h N + i and adding into forces F[h][N][3], so that the heads'
// force passes share one launch
template <int TPA, int BAS, bool VIR>
__global__ void __launch_bounds__(forces_threads<TPA>(), TPA >= 4 ? 4 : 1)
    k_forces(PairArgs a, const float *__restrict__ dpsi, float *__restrict__ F, float *__restrict__ vir_atom,
             int heads) {
    constexpr bool GS = forces_gsmem<TPA>();
    extern __shared__ __align__(16) float sbeta[];
    float *gsm = sbeta + a.S * a.S * NR * BETA_ROW;              // [atoms of the block][FG_ROW]
    stage_beta(a.beta, a.S, sbeta);
    griddep_wait();
    if (GS) {
        constexpr int APB = forces_threads<TPA>() / TPA;
        const int a_first = blockIdx.x * APB;
        // 16-byte loads: four consecutive components c..c+3 of one radial function s
        constexpr int V4 = NPSI / 4, C4 = NC / 4;
        for (int q = threadIdx.x; q < APB * V4; q += blockDim.x) {
            const int al = q / V4, e4 = q - al * V4, s = e4 / C4, c = 4 * (e4 - s * C4), m = a_first + al;
            const float4 v = m < a.N * heads ? __ldg(reinterpret_cast<const float4 *>(dpsi + (size_t)m * NPSI) + e4)
                                     : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            float *row = gsm + al * FG_ROW + c * 8 + s;
            row[0] = v.x;
            row[8] = v.y;
            row[16] = v.z;
            row[24] = v.w;
        }
    }
    __syncthreads();
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int atom_v = gt / TPA, sub = gt % TPA;
    const int head = a.N > 0 ? atom_v / a.N : 0, atom = atom_v - head * a.N;
    const bool active = atom_v < a.N * heads && !status_bad(a.status);
    F += (size_t)head * a.N * 3;
    float Fi[3] = {0.0f, 0.0f, 0.0f};
    float V[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) V[q] = 0.0f;
    if (active) {
        float g[GS ? 1 : NPSI];
        const float *gs = gsm + (threadIdx.x / TPA) * FG_ROW;
        if (!GS) {
            const float4 *g4 = reinterpret_cast<const float4 *>(dpsi + (size_t)atom_v * NPSI);
#pragma unroll
            for (int q = 0; q < NPSI / 4; ++q) {
                const float4 v = g4[q];
                g[4 * q] = v.x; g[4 * q + 1] = v.y; g[4 * q + 2] = v.z; g[4 * q + 3] = v.w;
            }
        }
        const int b = structure_of(a.atom_ptr, a.B, atom);
        const Centre ce(a, atom, b);
        const int zsi = clamp_species(a.species[atom], a.S, a.status);
        const float *brow = sbeta + zsi * a.S * (NR * BETA_ROW);
        const int p1 = a.row_ptr[atom + 1];
        PairPipe<1> pp(a, a.row_ptr[atom] + sub, p1, TPA);
        for (int p = a.row_ptr[atom] + sub; p < p1; p += TPA) {
            const NextPair cur = pp.next(a);
            if (!cur.ok) continue;
            const int j = cur.j;
            float fx, fy, fz;
            ce.displacement(cur, fx, fy, fz);
            float r, rinv;
            pair_length(fx, fy, fz, r, rinv);
            const float ux = fx * rinv, uy = fy * rinv, uz = fz * rinv;
            float B[NB], dB[NB];
            radial_basis<true, BAS>(a.rc, r, B, dB);
            float R[NR], Rp[NR];
            radial_combine<true>(brow + clamp_species(__float_as_int(cur.ph.w), a.S, a.status) * (NR * BETA_ROW), B,
                                 dB, R, Rp);
            float m[NC];
            monomials(ux, uy, uz, m);
            // One pass over the components: A_c = sum_s g_sc R_s, and per rank L the sums
            // P_L[s] = sum_(c of rank L) g_sc m_c.  Then
            //   S1 = sum_c A'_c m_c     = sum_s R'_s (P_0 + P_1 + P_2 + P_3)[s]
            //   S2 = sum_c L_c A_c m_c  = sum_s R_s (P_1 + 2 P_2 + 3 P_3)[s]
            //   Q  = sum_c A_c dm_c/du  = grad_u of the polynomial sum_c A_c m_c(u), in closed
            //        form for the rank-1, -2 and -3 monomials (~40 operations instead of 3 per
            //        component and the monomial derivatives)
            float A[NC], P[4][NR];
#pragma unroll
            for (int L = 0; L < 4; ++L)
#pragma unroll
                for (int s = 0; s < NR; ++s) P[L][s] = 0.0f;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                float gc[NR];
                if (GS) {
                    const float4 q4 = *reinterpret_cast<const float4 *>(gs + c * 8);
                    gc[0] = q4.x; gc[1] = q4.y; gc[2] = q4.z; gc[3] = q4.w;
                    gc[4] = gs[c * 8 + 4];
                } else {
#pragma unroll
                    for (int s = 0; s < NR; ++s) gc[s] = g[(GS ? 0 : s * NC + c)];
                }
                float Ac = 0.0f;
#pragma unroll
                for (int s = 0; s < NR; ++s) {
                    Ac = fmaf(gc[s], R[s], Ac);
                    P[comp_rank(c)][s] = fmaf(gc[s], m[c], P[comp_rank(c)][s]);
                }
                A[c] = Ac;
            }
            float S1 = 0.0f, S2 = 0.0f;
#pragma unroll
            for (int s = 0; s < NR; ++s) {
                S1 = fmaf(Rp[s], (P[0][s] + P[1][s]) + (P[2][s] + P[3][s]), S1);
                S2 = fmaf(R[s], fmaf(3.0f, P[3][s], fmaf(2.0f, P[2][s], P[1][s])), S2);
            }
            // components 4..9: xx xy xz yy yz zz; 10..19: xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
            const float xx = m[4], xy = m[5], xz = m[6], yy = m[7], yz = m[8], zz = m[9];
            float Q0 = A[1] + fmaf(2.0f * A[4], ux, fmaf(A[5], uy, A[6] * uz));
            float Q1 = A[2] + fmaf(A[5], ux, fmaf(2.0f * A[7], uy, A[8] * uz));
            float Q2 = A[3] + fmaf(A[6], ux, fmaf(A[8], uy, 2.0f * A[9] * uz));
            Q0 += fmaf(3.0f * A[10], xx, fmaf(2.0f * A[11], xy, fmaf(2.0f * A[12], xz,
                  fmaf(A[13], yy, fmaf(A[14], yz, A[15] * zz)))));
            Q1 += fmaf(A[11], xx, fmaf(2.0f * A[13], xy, fmaf(A[14], xz,
                  fmaf(3.0f * A[16], yy, fmaf(2.0f * A[17], yz, A[18] * zz)))));
            Q2 += fmaf(A[12], xx, fmaf(A[14], xy, fmaf(2.0f * A[15], xz,
                  fmaf(A[17], yy, fmaf(2.0f * A[18], yz, 3.0f * A[19] * zz)))));
            const float radial_term = S1 - S2 * rinv;
            const float gx = fmaf(ux, radial_term, Q0 * rinv);
            const float gy = fmaf(uy, radial_term, Q1 * rinv);
            const float gz = fmaf(uz, radial_term, Q2 * rinv);
            Fi[0] += gx; Fi[1] += gy; Fi[2] += gz;
            atomicAdd(F + 3 * j, -gx);
            atomicAdd(F + 3 * j + 1, -gy);
            atomicAdd(F + 3 * j + 2, -gz);
            if (VIR) {
                V[0] -= fx * gx; V[1] -= fx * gy; V[2] -= fx * gz;
                V[3] -= fy * gx; V[4] -= fy * gy; V[5] -= fy * gz;
                V[6] -= fz * gx; V[7] -= fz * gy; V[8] -= fz * gz;
            }
        }
    }
    if (TPA > 1) {
#pragma unroll
        for (int off = TPA / 2; off > 0; off >>= 1) {
#pragma unroll
            for (int q = 0; q < 3; ++q) Fi[q] += __shfl_xor_sync(0xffffffffu, Fi[q], off);
            if (VIR) {
#pragma unroll
                for (int q = 0; q < 9; ++q) V[q] += __shfl_xor_sync(0xffffffffu, V[q], off);
            }
        }
    }
    if (!active || sub != 0) return;
    atomicAdd(F + 3 * atom, Fi[0]);
    atomicAdd(F + 3 * atom + 1, Fi[1]);
    atomicAdd(F + 3 * atom + 2, Fi[2]);
    if (VIR) {
#pragma unroll
        for (int q = 0; q < 9; ++q) vir_atom[(size_t)atom * 9 + q] = V[q];
    }
}

// Tangent moments for the parameter gradient: dPsi_i/dt when every position moves along
// v (= dL/dF), i.e. d_ij changes by v_j - v_i.  Per pair and component c of rank L:
//   d/dt [R_s m_c] = R'_s w m_c + R_s (D_c - L_c m_c w) / r,  w = u . dd,  D_c = dd . dm_c/du.
template <int TPA, int BAS>
__global__ void __launch_bounds__(256) k_moments_tangent(PairArgs a, const float *__restrict__ vel,
                                                         float *__restrict__ psid) {
    extern __shared__ __align__(16) float sbeta[];
    stage_beta(a.beta, a.S, sbeta);
    griddep_wait();
    __syncthreads();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int atom = g / TPA, sub = g % TPA;
    const bool active = atom < a.N && !status_bad(a.status);
    float acc[NPSI];
#pragma unroll
    for (int q = 0; q < NPSI; ++q) acc[q] = 0.0f;
    if (active) {
        const int b = structure_of(a.atom_ptr, a.B, atom);
        const Centre ce(a, atom, b);
        const float vix = vel[3 * atom], viy = vel[3 * atom + 1], viz = vel[3 * atom + 2];
        const int zsi = clamp_species(a.species[atom], a.S, a.status);
        const float *brow = sbeta + zsi * a.S * (NR * BETA_ROW);
        const int p1 = a.row_ptr[atom + 1];
        PairPipe<1> pp(a, a.row_ptr[atom] + sub, p1, TPA, vel);
        for (int p = a.row_ptr[atom] + sub; p < p1; p += TPA) {
            const NextPair cur = pp.next(a);
            if (!cur.ok) continue;
            float fx, fy, fz;
            ce.displacement(cur, fx, fy, fz);
            float r, rinv;
            pair_length(fx, fy, fz, r, rinv);
            const float ux = fx * rinv, uy = fy * rinv, uz = fz * rinv;
            const float ddx = cur.vx - vix, ddy = cur.vy - viy, ddz = cur.vz - viz;
            const float w = ux * ddx + uy * ddy + uz * ddz;
            float B[NB], dB[NB];
            radial_basis<true, BAS>(a.rc, r, B, dB);
            float R[NR], Rp[NR];
            radial_combine<true>(brow + clamp_species(__float_as_int(cur.ph.w), a.S, a.status) * (NR * BETA_ROW), B,
                                 dB, R, Rp);
#pragma unroll
            for (int s = 0; s < NR; ++s) Rp[s] *= w;
            float m[NC];
            monomials(ux, uy, uz, m);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const float Dc = ddx * dmono(c, 0, ux, uy, uz) + ddy * dmono(c, 1, ux, uy, uz) +
                                 ddz * dmono(c, 2, ux, uy, uz);
                const float ang = (Dc - (float)comp_rank(c) * m[c] * w) * rinv;
#pragma unroll
                for (int s = 0; s < NR; ++s) acc[s * NC + c] = fmaf(Rp[s], m[c], fmaf(R[s], ang, acc[s * NC + c]));
            }
        }
    }
    if (TPA > 1) {
#pragma unroll
        for (int off = TPA / 2; off > 0; off >>= 1)
#pragma unroll
            for (int q = 0; q < NPSI; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
    }
    if (!active) return;
    float *out = psid + (size_t)atom * NPSI;
#pragma unroll
    for (int q = 0; q < NPSI; ++q)
        if (q % TPA == sub) out[q] = acc[q];
}

// Species-pair coefficient gradient.  With psib = dJ/dPsi and psidb = dJ/dPsid of atom i,
// per pair and radial function s (coefficients pre-scaled by n_basis^{-1/2}):
//   dJ/dbeta[zi][zj][s][k] += B_k (P1_s + P3_s / r) + B'_k w P2_s
//   P1_s = sum_c psib[s][c] m_c,  P2_s = sum_c psidb[s][c] m_c,
//   P3_s = sum_c psidb[s][c] (D_c - L_c m_c w)
// accumulated per block in shared memory, block partials written to part[block][S S 35].
// dJ/dbeta partials.  One warp per centre atom i (species zi); each lane accumulates its pairs'
// NR x NB terms B_k alpha_s + dB_k gamma_s into its own slice of shared memory, indexed by the
// neighbour's species (layout [z][s][k][lane]: lanes never share a bank, no atomics).  A warp
// takes its atoms 32 at a time, species by species: after the rows of one centre species the
// lanes add up the 32 slices (lane l takes entries l, l + 32, ...) into the block's
// [S][S][NR][NB] accumulator (one atomic per entry, distinct entries per lane) and clear
// them.  Block partials are summed in a fixed order by k_pg_beta_reduce.
template <int BAS>
__global__ void __launch_bounds__(256) k_pg_beta(PairArgs a, const float *__restrict__ vel,
                                                 const float *__restrict__ psib, const float *__restrict__ psidb,
                                                 float *__restrict__ part) {
    extern __shared__ float sm[];
    const int nbeta = a.S * a.S * NR * NB, nlane = a.S * NR * NB;     // per-lane slice: [S][NR][NB]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    float *acc = sm;                                                   // [nbeta]
    float *pw = sm + nbeta + warp * 2 * NPSI;                          // this warp's psib, psidb
    float *la = sm + nbeta + nwarps * 2 * NPSI + (size_t)warp * nlane * 32;
    for (int q = threadIdx.x; q < nbeta; q += blockDim.x) acc[q] = 0.0f;
    for (int q = lane; q < nlane * 32; q += 32) la[q] = 0.0f;
    __syncthreads();
    const bool ok_status = !status_bad(a.status);
    const unsigned full = 0xffffffffu;
    const int gw = blockIdx.x * nwarps + warp, nwt = gridDim.x * nwarps;
    for (int g0 = gw; ok_status && g0 < a.N; g0 += 32 * nwt) {
      const int mine = g0 + lane * nwt;                          // this lane's atom of the group
      const int zmine = mine < a.N ? clamp_species(a.species[mine], a.S, a.status) : -1;
      for (int zsi = 0; zsi < a.S; ++zsi) {
        unsigned todo = __ballot_sync(full, zmine == zsi);
        if (!todo) continue;
        while (todo) {
        const int atom = g0 + (__ffs(todo) - 1) * nwt;
        todo &= todo - 1u;
        for (int q = lane; q < NPSI; q += 32) {
            pw[q] = psib[(size_t)atom * NPSI + q];
            pw[NPSI + q] = psidb[(size_t)atom * NPSI + q];
        }
        __syncwarp();
        const int b = structure_of(a.atom_ptr, a.B, atom);
        const Centre ce(a, atom, b);
        const float vix = vel[3 * atom], viy = vel[3 * atom + 1], viz = vel[3 * atom + 2];
        const int p1 = a.row_ptr[atom + 1];
        PairPipe<1> pp(a, a.row_ptr[atom] + lane, p1, 32, vel);
        for (int p = a.row_ptr[atom] + lane; p < p1; p += 32) {
            const NextPair cur = pp.next(a);
            if (!cur.ok) continue;
            float fx, fy, fz;
            ce.displacement(cur, fx, fy, fz);
            float r, rinv;
            pair_length(fx, fy, fz, r, rinv);
            const float ux = fx * rinv, uy = fy * rinv, uz = fz * rinv;
            const float ddx = cur.vx - vix, ddy = cur.vy - viy, ddz = cur.vz - viz;
            const float w = ux * ddx + uy * ddy + uz * ddz;
            float B[NB], dB[NB];
            radial_basis<true, BAS>(a.rc, r, B, dB);
            float m[NC], ang[NC];
            monomials(ux, uy, uz, m);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const float Dc = ddx * dmono(c, 0, ux, uy, uz) + ddy * dmono(c, 1, ux, uy, uz) +
                                 ddz * dmono(c, 2, ux, uy, uz);
                ang[c] = Dc - (float)comp_rank(c) * m[c] * w;
            }
            float *dst = la + (size_t)clamp_species(__float_as_int(cur.ph.w), a.S, a.status) * (NR * NB) * 32 + lane;
#pragma unroll
            for (int s = 0; s < NR; ++s) {
                float P1 = 0.0f, P2 = 0.0f, P3 = 0.0f;
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    P1 = fmaf(pw[s * NC + c], m[c], P1);
                    P2 = fmaf(pw[NPSI + s * NC + c], m[c], P2);
                    P3 = fmaf(pw[NPSI + s * NC + c], ang[c], P3);
                }
                const float alpha = fmaf(P3, rinv, P1), gam = w * P2;
#pragma unroll
                for (int k = 0; k < NB; ++k) dst[(s * NB + k) * 32] += fmaf(B[k], alpha, dB[k] * gam);
            }
        }
        __syncwarp();
        }
        // add the lanes' slices into the block accumulator for species row zi, and clear them
        for (int e = lane; e < nlane; e += 32) {
            float t = 0.0f;
            float *row = la + (size_t)e * 32;
#pragma unroll 8
            for (int l = 0; l < 32; ++l) {                         // rotated: lanes read distinct banks
                const int ll = (l + lane) & 31;
                t += row[ll];
                row[ll] = 0.0f;
            }
            if (t != 0.0f) atomicAdd(acc + zsi * nlane + e, t);
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nbeta; q += blockDim.x) part[(size_t)blockIdx.x * nbeta + q] = acc[q];
}

// shared memory of the staged coefficient rows (61 KB for 16 species: above the default
// 48 KB, so the kernels opt in once)
static size_t beta_smem_bytes(int S) { return sizeof(float) * (size_t)S * S * NR * BETA_ROW; }
template <typename Kern>
static void allow_beta_smem(Kern kernel, size_t extra = 0) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(beta_smem_bytes(MAX_S) + extra));
}

// 2 and 4 lanes per atom take the component-split kernel, the others k_moments
template <int TPA, int BAS>
static void launch_moments_t(const PairArgs &a, float *psi, cudaStream_t st) {
    constexpr bool CS = TPA == 2 || TPA == 4;
    const int threads = CS ? 256 : moments_threads<TPA>();
    const long long total = (long long)a.N * TPA;
    const int blocks = (int)((total + threads - 1) / threads);
    const size_t smem = beta_smem_bytes(a.S);
    auto kern = CS ? k_moments_cs<(CS ? TPA : 2), BAS> : k_moments<TPA, BAS>;
    static PerDeviceOnce attr;
    if (attr.first()) {
        allow_beta_smem(kern);
    }
    if (blocks > 0) {
        launch_pdl(kern, dim3(blocks), dim3(threads), smem, st, a, psi);
        note_launches(1);
    }
}

template <int TPA, int BAS>
static void launch_forces_t(const PairArgs &a, const float *dpsi, float *F, float *vir, cudaStream_t st,
                            int heads) {
    const int threads = forces_threads<TPA>();
    const long long total = (long long)a.N * heads * TPA;
    const int blocks = (int)((total + threads - 1) / threads);
    const size_t smem = beta_smem_bytes(a.S) +
                        (forces_gsmem<TPA>() ? sizeof(float) * (threads / TPA) * FG_ROW : 0);
    auto kern = vir ? k_forces<TPA, BAS, true> : k_forces<TPA, BAS, false>;
    static PerDeviceOnce attr;
    if (attr.first()) {
        const size_t extra = forces_gsmem<TPA>() ? sizeof(float) * (threads / TPA) * FG_ROW : 0;
        allow_beta_smem(k_forces<TPA, BAS, true>, extra);
        allow_beta_smem(k_forces<TPA, BAS, false>, extra);
    }
    if (blocks > 0) {
        launch_pdl(kern, dim3(blocks), dim3(threads), smem, st, a, dpsi, F, vir, heads);
        note_launches(1);
    }
}

template <int BAS>
static void launch_moments_b(const PairArgs &a, int tpa, float *psi, cudaStream_t st) {
    switch (tpa) {
    case 1: launch_moments_t<1, BAS>(a, psi, st); break;
    case 2: launch_moments_t<2, BAS>(a, psi, st); break;
    case 4: launch_moments_t<4, BAS>(a, psi, st); break;
    case 8: launch_moments_t<8, BAS>(a, psi, st); break;
    case 16: launch_moments_t<16, BAS>(a, psi, st); break;
    default: launch_moments_t<32, BAS>(a, psi, st); break;
    }
}

void launch_moments(const PairArgs &a, int tpa, float *psi, cudaStream_t st) {
    if (a.rc.basis == BASIS_BESSEL) launch_moments_b<BASIS_BESSEL>(a, tpa, psi, st);
    else launch_moments_b<BASIS_GAUSSIAN>(a, tpa, psi, st);
}

template <int BAS>
static void launch_forces_b(const PairArgs &a, int tpa, const float *dpsi, float *F, float *vir, cudaStream_t st,
                            int heads) {
    switch (tpa) {
    case 1: launch_forces_t<1, BAS>(a, dpsi, F, vir, st, heads); break;
    case 2: launch_forces_t<2, BAS>(a, dpsi, F, vir, st, heads); break;
    case 4: launch_forces_t<4, BAS>(a, dpsi, F, vir, st, heads); break;
    case 8: launch_forces_t<8, BAS>(a, dpsi, F, vir, st, heads); break;
    case 16: launch_forces_t<16, BAS>(a, dpsi, F, vir, st, heads); break;
    default: launch_forces_t<32, BAS>(a, dpsi, F, vir, st, heads); break;
    }
}

void launch_forces(const PairArgs &a, int tpa, const float *dpsi, float *F, float *vir, cudaStream_t st, int heads) {
    if (heads < 1 || (heads > 1 && vir)) return;                    // heads: no virial
    if (a.rc.basis == BASIS_BESSEL) launch_forces_b<BASIS_BESSEL>(a, tpa, dpsi, F, vir, st, heads);
    else launch_forces_b<BASIS_GAUSSIAN>(a, tpa, dpsi, F, vir, st, heads);
}

}  // namespace gm

namespace gm {

template <int TPA, int BAS>
static void launch_tangent_t(const PairArgs &a, const float *vel, float *psid, cudaStream_t st) {
    const int threads = 256;
    const long long total = (long long)a.N * TPA;
    const int blocks = (int)((total + threads - 1) / threads);
    const size_t smem = beta_smem_bytes(a.S);
    static PerDeviceOnce attr;
    if (attr.first()) {
        allow_beta_smem(k_moments_tangent<TPA, BAS>);
    }
    if (blocks > 0) {
        launch_pdl(k_moments_tangent<TPA, BAS>, dim3(blocks), dim3(threads), smem, st, a, vel, psid);
        note_launches(1);
    }
}

template <int BAS>
static void launch_tangent_b(const PairArgs &a, int tpa, const float *vel, float *psid, cudaStream_t st) {
    switch (tpa) {
    case 1: launch_tangent_t<1, BAS>(a, vel, psid, st); break;
    case 2: launch_tangent_t<2, BAS>(a, vel, psid, st); break;
    case 4: launch_tangent_t<4, BAS>(a, vel, psid, st); break;
    case 8: launch_tangent_t<8, BAS>(a, vel, psid, st); break;
    case 16: launch_tangent_t<16, BAS>(a, vel, psid, st); break;
    default: launch_tangent_t<32, BAS>(a, vel, psid, st); break;
    }
}

void launch_moments_tangent(const PairArgs &a, int tpa, const float *vel, float *psid, cudaStream_t st) {
    if (a.rc.basis == BASIS_BESSEL) launch_tangent_b<BASIS_BESSEL>(a, tpa, vel, psid, st);
    else launch_tangent_b<BASIS_GAUSSIAN>(a, tpa, vel, psid, st);
}

// warps per block of k_pg_beta: the per-lane slices take S x NR x NB x 32 floats per warp
static int pg_beta_warps(int S) {
    const size_t per_warp = sizeof(float) * ((size_t)S * NR * NB * 32 + 2 * NPSI);
    int w = (int)((96u << 10) / per_warp);
    return w < 1 ? 1 : (w > 8 ? 8 : w);
}

int pg_beta_blocks(int N, int S) {
    const int w = pg_beta_warps(S);
    const int b = (N + w - 1) / w;
    return b < 1 ? 1 : (b > 148 * 2 ? 148 * 2 : b);
}

void launch_pg_beta(const PairArgs &a, const float *vel, const float *psib, const float *psidb, float *part,
                    cudaStream_t st) {
    const int w = pg_beta_warps(a.S);
    const int blocks = pg_beta_blocks(a.N, a.S);
    const size_t smem = sizeof(float) * ((size_t)a.S * a.S * NR * NB + (size_t)w * (2 * NPSI + a.S * NR * NB * 32));
    if (a.N > 0) {
        if (a.rc.basis == BASIS_BESSEL) {
            cudaFuncSetAttribute(k_pg_beta<BASIS_BESSEL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_pg_beta<BASIS_BESSEL><<<blocks, 32 * w, smem, st>>>(a, vel, psib, psidb, part);
        } else {
            cudaFuncSetAttribute(k_pg_beta<BASIS_GAUSSIAN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_pg_beta<BASIS_GAUSSIAN><<<blocks, 32 * w, smem, st>>>(a, vel, psib, psidb, part);
        }
        note_launches(1);
    }
}

}  // namespace gm
