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
// Pipeline (all on one stream, no host synchronisation):
//   setup    per-structure cell grid (cells >= r_cut, at most max(1, n_atoms) cells)
//   bin      wrap positions, cell index, atomic histogram
//   scan     cell offsets
//   scatter  atoms into cells (atomic slots); sortcells (one warp per cell) packs each
//            cell's FP32 wrapped positions in ascending atom index (float4, index in w)
//   search   one warp per atom: count pass -> scan -> row_ptr -> fill pass (same order)
#include <math.h>

#include <optional>

#include "gm_internal.h"

namespace gm {

// ------------------------------------------------------------------ scan
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_BLOCK = SCAN_THREADS * 4;

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_local(const int32_t *__restrict__ in, int32_t *out, int n,
                                                             int32_t *block_sums) {
    __shared__ int32_t s[SCAN_THREADS];
    const int t = threadIdx.x;
    const int base = blockIdx.x * SCAN_BLOCK + t * 4;
    int v[4], sum = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v[q] = (base + q < n) ? in[base + q] : 0;
        sum += v[q];
    }
    s[t] = sum;
    __syncthreads();
    for (int off = 1; off < SCAN_THREADS; off <<= 1) {
        int x = t >= off ? s[t - off] : 0;
        __syncthreads();
        s[t] += x;
        __syncthreads();
    }
    int excl = s[t] - sum;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (base + q < n) out[base + q] = excl;
        excl += v[q];
    }
    if (t == SCAN_THREADS - 1) block_sums[blockIdx.x] = s[t];
}

__global__ void __launch_bounds__(1024) k_scan_sums(int32_t *block_sums, int nb, int32_t *total_out) {
    __shared__ int32_t s[1024];
    __shared__ int32_t carry;
    const int t = threadIdx.x;
    if (t == 0) carry = 0;
    __syncthreads();
    for (int chunk = 0; chunk < nb; chunk += 1024) {
        const int idx = chunk + t;
        const int v = idx < nb ? block_sums[idx] : 0;
        s[t] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            int x = t >= off ? s[t - off] : 0;
            __syncthreads();
            s[t] += x;
            __syncthreads();
        }
        if (idx < nb) block_sums[idx] = carry + s[t] - v;
        __syncthreads();
        if (t == 1023) carry += s[1023];
        __syncthreads();
    }
    if (t == 0) *total_out = carry;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_add(int32_t *out, int n, const int32_t *__restrict__ block_sums) {
    const int add = block_sums[blockIdx.x];
    const int base = blockIdx.x * SCAN_BLOCK + threadIdx.x * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (base + q < n) out[base + q] += add;
}

size_t scan_tmp_ints(int n) { return (size_t)((n + SCAN_BLOCK - 1) / SCAN_BLOCK) + 1; }

void exclusive_scan(const int32_t *in, int32_t *out, int n, int32_t *tmp, cudaStream_t st) {
    const int nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
    if (nb > 0) k_scan_local<<<nb, SCAN_THREADS, 0, st>>>(in, out, n, tmp);
    k_scan_sums<<<1, 1024, 0, st>>>(tmp, nb, out + n);
    if (nb > 0) k_scan_add<<<nb, SCAN_THREADS, 0, st>>>(out, n, tmp);
    note_launches(nb > 0 ? 3 : 1);
}

// ------------------------------------------------------------------ setup
__global__ void __launch_bounds__(1024) k_nl_setup(int B, const int32_t *__restrict__ atom_ptr,
                                                   const double *__restrict__ cell, const uint8_t *__restrict__ pbc,
                                                   double rc, NlStruct *S, int32_t *status) {
    __shared__ int32_t s[1024];
    __shared__ int32_t carry;
    const int t = threadIdx.x;
    if (t == 0) carry = 0;
    __syncthreads();
    for (int chunk = 0; chunk < B; chunk += 1024) {
        const int b = chunk + t;
        NlStruct q;
        int ncell = 0;
        if (b < B) {
            const double *C = cell + 9 * b;
            const bool ortho = C[1] == 0.0 && C[2] == 0.0 && C[3] == 0.0 && C[5] == 0.0 && C[6] == 0.0 && C[7] == 0.0;
            const bool periodic = pbc[3 * b] && pbc[3 * b + 1] && pbc[3 * b + 2];
            const bool positive = C[0] > 0.0 && C[4] > 0.0 && C[8] > 0.0;
            q.a0 = atom_ptr[b];
            q.n = atom_ptr[b + 1] - q.a0;
            bool ok = ortho && periodic && positive;
            long long nc[3];
            for (int a = 0; a < 3; ++a) {
                q.L[a] = ok ? C[4 * a] : 1.0;
                double f = floor(q.L[a] / (rc * (1.0 + 1e-5)));
                nc[a] = f < 1.0 ? 1 : (f > 1024.0 ? 1024 : (long long)f);
            }
            const long long limit = q.n > 1 ? q.n : 1;
            while (nc[0] * nc[1] * nc[2] > limit) {
                int am = 0;
                if (nc[1] > nc[am]) am = 1;
                if (nc[2] > nc[am]) am = 2;
                nc[am] -= 1;
            }
            int Kmax = 0;
            double Lmax = 0.0;
            for (int a = 0; a < 3; ++a) {
                q.nc[a] = (int)nc[a];
                q.cs[a] = q.L[a] / (double)nc[a];
                int K = (int)ceil(rc / q.cs[a] + 1e-6);
                if (K > 100) { ok = false; K = 0; }
                q.K[a] = ok ? K : 0;
                q.Lf[a] = (float)q.L[a];
                Kmax = K > Kmax ? K : Kmax;
                Lmax = q.L[a] > Lmax ? q.L[a] : Lmax;
            }
            if (!ok) set_status(status, GM_ERR_UNSUPPORTED);
            // |FP32 displacement error| per axis <= 2^-24 L (6 + 2K); bound r^2 error near r_cut
            const double u = 5.9604644775390625e-8;  // 2^-24
            const double e = u * Lmax * (8.0 + 4.0 * Kmax);
            q.eps2 = (float)(4.0 * (2.0 * 1.7320508075688772 * e * rc + 3.0 * e * e + 4.0 * u * rc * rc) + 1e-30);
            ncell = q.nc[0] * q.nc[1] * q.nc[2];
        }
        s[t] = ncell;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            int x = t >= off ? s[t - off] : 0;
            __syncthreads();
            s[t] += x;
            __syncthreads();
        }
        if (b < B) {
            q.cell0 = carry + s[t] - ncell;
            S[b] = q;
        }
        __syncthreads();
        if (t == 1023) carry += s[1023];
        __syncthreads();
    }
}

// ------------------------------------------------------------------ bin
// Wrap of one coordinate; the same correctly rounded sequence as the oracle.
__device__ __forceinline__ double wrap_axis(double x, double L, int &m_out) {
    double m = floor(__ddiv_rn(x, L));
    double xw = __dsub_rn(x, __dmul_rn(m, L));
    if (xw < 0.0) { m -= 1.0; xw = __dsub_rn(x, __dmul_rn(m, L)); }
    if (xw >= L) { m += 1.0; xw = __dsub_rn(x, __dmul_rn(m, L)); }
    if (xw < 0.0 || xw >= L) xw = 0.0;
    m_out = (fabs(m) < 1.0e6) ? (int)m : 0;
    return xw;
}

__global__ void __launch_bounds__(256) k_nl_bin(int N, int B, const int32_t *__restrict__ atom_ptr,
                                                const double *__restrict__ pos, const int32_t *__restrict__ species,
                                                int n_species, const NlStruct *__restrict__ S, int32_t *sid, double *xw,
                                                int32_t *mimg, int32_t *cellid, int32_t *ccount, int32_t *status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int b = structure_of(atom_ptr, B, i);
    sid[i] = b;
    const int z = species[i];
    if (z < 0 || z >= n_species) set_status(status, GM_ERR_SPECIES);
    const NlStruct &q = S[b];
    int ic[3];
    for (int a = 0; a < 3; ++a) {
        const double x = pos[3 * i + a];
        int m;
        const double w = wrap_axis(x, q.L[a], m);
        if (!(fabs(x) < 1.0e6 * q.L[a])) set_status(status, GM_ERR_UNSUPPORTED);
        xw[3 * i + a] = w;
        mimg[3 * i + a] = m;
        int c = (int)floor(__ddiv_rn(w, q.cs[a]));
        c = c < 0 ? 0 : (c >= q.nc[a] ? q.nc[a] - 1 : c);
        ic[a] = c;
    }
    const int cid = q.cell0 + (ic[2] * q.nc[1] + ic[1]) * q.nc[0] + ic[0];
    cellid[i] = cid;
    atomicAdd(ccount + cid, 1);
}

__global__ void __launch_bounds__(256) k_nl_scatter(int N, const int32_t *__restrict__ cellid,
                                                    const int32_t *__restrict__ cstart, int32_t *cfill, int32_t *sorted) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int c = cellid[i];
    const int slot = atomicAdd(cfill + c, 1);
    sorted[cstart[c] + slot] = i;
}

// One warp per cell: each atom's position in the cell is its rank among the cell's atom
// indices (all distinct), so the packed order is ascending atom index (deterministic).
__global__ void __launch_bounds__(256) k_nl_sortcells(int ncells, const int32_t *__restrict__ cstart,
                                                      const int32_t *__restrict__ unsorted,
                                                      const double *__restrict__ xw, float4 *xs) {
    const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= ncells) return;
    const int s0 = cstart[c], n = cstart[c + 1] - s0;
    for (int e = lane; e < n; e += 32) {
        const int v = unsorted[s0 + e];
        int r = 0;
        for (int q = 0; q < n; ++q) r += unsorted[s0 + q] < v;
        xs[s0 + r] = make_float4((float)xw[3 * v], (float)xw[3 * v + 1], (float)xw[3 * v + 2], __int_as_float(v));
    }
}

__device__ __forceinline__ int floordiv(int v, int n) { return v >= 0 ? v / n : -((-v + n - 1) / n); }

// ------------------------------------------------------------------ search
// G lanes per centre atom (atoms taken in cell order for locality; G = 32 for small
// systems, 8 for large ones, whose cells hold about 20 candidates); lanes test G
// candidates of a cell at a time.  The fill pass places accepted pairs with a ballot over
// the group, so the row order is the candidate order (stencil cell, then ascending
// neighbour index) in both passes.
template <bool FILL, int G>
__global__ void __launch_bounds__(256) k_nl_search(int N, const NlStruct *__restrict__ S, const int32_t *__restrict__ sid,
                                                   const int32_t *__restrict__ cellid, const int32_t *__restrict__ cstart,
                                                   const float4 *__restrict__ xs, const double *__restrict__ xw,
                                                   const int32_t *__restrict__ mimg, double rc, float rc2f,
                                                   int32_t *counts, const int32_t *__restrict__ row_ptr, int64_t cap,
                                                   int32_t *col, char4 *shift, int32_t *status) {
    // G lanes per centre atom (G = 8 or 32); the ballots below involve only the group
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int lane = threadIdx.x % G;
    constexpr unsigned low_mask = (G == 32) ? 0xffffffffu : ((1u << (G % 32)) - 1u);
    const int group_shift = (threadIdx.x & 31) & ~(G - 1);
    const unsigned group_mask = low_mask << group_shift;
    const int t = gid;
    if (t >= N) return;
    if (FILL) {
        if ((int64_t)row_ptr[N] > cap) return;
        if (status_bad(status)) return;
    }
    const float4 me = xs[t];
    const int i = __float_as_int(me.w);
    const NlStruct &q = S[sid[i]];
    const int cid = cellid[i] - q.cell0;
    const int ix = cid % q.nc[0], iy = (cid / q.nc[0]) % q.nc[1], iz = cid / (q.nc[0] * q.nc[1]);
    const double rc2 = __dmul_rn(rc, rc);
    const float lo = rc2f - q.eps2, hi = rc2f + q.eps2;
    const int mi0 = mimg[3 * i], mi1 = mimg[3 * i + 1], mi2 = mimg[3 * i + 2];
    const double xi0 = xw[3 * i], xi1 = xw[3 * i + 1], xi2 = xw[3 * i + 2];
    const unsigned below = (1u << lane) - 1u;
    int out = FILL ? row_ptr[i] : 0;
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
                const int k0 = cstart[c], k1 = cstart[c + 1];
                for (int base = k0; base < k1; base += G) {
                    const int k = base + lane;
                    bool in = false;
                    int j = 0;
                    if (k < k1) {
                        const float4 o = xs[k];
                        j = __float_as_int(o.w);
                        if (!(zero_shift && j == i)) {
                            const float fx = (o.x - me.x) + sx, fy = (o.y - me.y) + sy, fz = (o.z - me.z) + sz;
                            const float r2 = fx * fx + fy * fy + fz * fz;
                            if (r2 < lo) in = true;
                            else if (r2 <= hi) {
                                const double d0 = __dadd_rn(__dsub_rn(xw[3 * j], xi0), __dmul_rn((double)nx, q.L[0]));
                                const double d1 = __dadd_rn(__dsub_rn(xw[3 * j + 1], xi1), __dmul_rn((double)ny, q.L[1]));
                                const double d2 = __dadd_rn(__dsub_rn(xw[3 * j + 2], xi2), __dmul_rn((double)nz, q.L[2]));
                                const double r2d =
                                    __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
                                in = r2d < rc2;
                            }
                        }
                    }
                    const unsigned ball = (__ballot_sync(group_mask, in) >> group_shift) & low_mask;
                    if (FILL) {
                        if (in) {
                            const int pos = out + __popc(ball & below);
                            const int s0 = nx - mimg[3 * j] + mi0;
                            const int s1 = ny - mimg[3 * j + 1] + mi1;
                            const int s2 = nz - mimg[3 * j + 2] + mi2;
                            if (s0 < -127 || s0 > 127 || s1 < -127 || s1 > 127 || s2 < -127 || s2 > 127)
                                set_status(status, GM_ERR_UNSUPPORTED);
                            col[pos] = j;
                            shift[pos] = make_char4((signed char)s0, (signed char)s1, (signed char)s2, 0);
                        }
                        out += __popc(ball);
                    } else {
                        cnt += __popc(ball);
                    }
                }
            }
        }
    }
    if (!FILL && lane == 0) counts[i] = cnt;
}

__global__ void k_nl_total(const int32_t *__restrict__ rowN, int64_t cap, int64_t *n_pairs, int32_t *status) {
    const int64_t P = *rowN;
    *n_pairs = P;
    if (P > cap) set_status(status, GM_ERR_CAPACITY);
}

// ------------------------------------------------------------------ host
struct NlWs {
    NlStruct *S;
    int32_t *sid, *mimg, *cellid, *ccount, *cstart, *cfill, *unsorted, *counts, *scan_tmp;
    double *xw;
    float4 *xs;
};

static NlWs carve_nl(Carve &c, int B, int N) {
    NlWs w;
    const int ncmax = N + B;
    const size_t n1 = N > 0 ? (size_t)N : 1;
    w.S = c.take<NlStruct>(B);
    w.sid = c.take<int32_t>(n1);
    w.xw = c.take<double>(3 * n1);
    w.mimg = c.take<int32_t>(3 * n1);
    w.cellid = c.take<int32_t>(n1);
    w.ccount = c.take<int32_t>(ncmax);
    w.cstart = c.take<int32_t>(ncmax + 1);
    w.cfill = c.take<int32_t>(ncmax);
    w.unsorted = c.take<int32_t>(n1);
    w.xs = c.take<float4>(n1);
    w.counts = c.take<int32_t>(n1);
    w.scan_tmp = c.take<int32_t>(scan_tmp_ints(ncmax + 1 > N ? ncmax + 1 : N));
    return w;
}

size_t nl_workspace_bytes(int n_struct, int n_atoms) {
    Carve c(reinterpret_cast<void *>(256), ~size_t(0) >> 1);
    carve_nl(c, n_struct, n_atoms);
    return c.off + 256;
}

gm_status nl_build(const gm_system &sys, double r_cut, int n_species, gm_nlist &nl, void *ws, size_t ws_bytes,
                   int32_t *status, cudaStream_t st) {
    const int B = sys.n_structures, N = sys.n_atoms;
    Carve c(ws, ws_bytes);
    NlWs w = carve_nl(c, B, N);
    if (!c.ok) return GM_ERR_WORKSPACE;
    const int ncmax = N + B;
    std::optional<StageScope> scope;  // sub-stage events (profiling only)
    scope.emplace(ST_NL_BIN, st);
    if (cudaMemsetAsync(w.ccount, 0, sizeof(int32_t) * ncmax, st) != cudaSuccess) return GM_ERR_CUDA;
    if (cudaMemsetAsync(w.cfill, 0, sizeof(int32_t) * ncmax, st) != cudaSuccess) return GM_ERR_CUDA;
    k_nl_setup<<<1, 1024, 0, st>>>(B, sys.atom_ptr, sys.cell, sys.pbc, r_cut, w.S, status);
    note_launches(1);
    const int tb = 256;
    if (N > 0) {
        k_nl_bin<<<(N + tb - 1) / tb, tb, 0, st>>>(N, B, sys.atom_ptr, sys.pos, sys.species, n_species, w.S, w.sid,
                                                   w.xw, w.mimg, w.cellid, w.ccount, status);
        note_launches(1);
    }
    exclusive_scan(w.ccount, w.cstart, ncmax, w.scan_tmp, st);
    if (N > 0) {
        k_nl_scatter<<<(N + tb - 1) / tb, tb, 0, st>>>(N, w.cellid, w.cstart, w.cfill, w.unsorted);
        const int G = N >= 16384 ? 8 : 32;
        const long long warps_cells = (long long)ncmax * 32, warps_atoms = (long long)N * G;
        k_nl_sortcells<<<(int)((warps_cells + tb - 1) / tb), tb, 0, st>>>(ncmax, w.cstart, w.unsorted, w.xw, w.xs);
        const float rc2f = (float)(r_cut * r_cut);
        scope.reset();
        scope.emplace(ST_NL_COUNT, st);
        if (G == 8)
            k_nl_search<false, 8><<<(int)((warps_atoms + tb - 1) / tb), tb, 0, st>>>(
                N, w.S, w.sid, w.cellid, w.cstart, w.xs, w.xw, w.mimg, r_cut, rc2f, w.counts, nullptr, 0, nullptr,
                nullptr, status);
        else
            k_nl_search<false, 32><<<(int)((warps_atoms + tb - 1) / tb), tb, 0, st>>>(
                N, w.S, w.sid, w.cellid, w.cstart, w.xs, w.xw, w.mimg, r_cut, rc2f, w.counts, nullptr, 0, nullptr,
                nullptr, status);
        scope.reset();
        scope.emplace(ST_NL_SCAN, st);
        exclusive_scan(w.counts, nl.row_ptr, N, w.scan_tmp, st);
        k_nl_total<<<1, 1, 0, st>>>(nl.row_ptr + N, nl.capacity, nl.n_pairs, status);
        scope.reset();
        scope.emplace(ST_NL_FILL, st);
        if (G == 8)
            k_nl_search<true, 8><<<(int)((warps_atoms + tb - 1) / tb), tb, 0, st>>>(
                N, w.S, w.sid, w.cellid, w.cstart, w.xs, w.xw, w.mimg, r_cut, rc2f, nullptr, nl.row_ptr, nl.capacity,
                nl.col, reinterpret_cast<char4 *>(nl.shift), status);
        else
            k_nl_search<true, 32><<<(int)((warps_atoms + tb - 1) / tb), tb, 0, st>>>(
                N, w.S, w.sid, w.cellid, w.cstart, w.xs, w.xw, w.mimg, r_cut, rc2f, nullptr, nl.row_ptr, nl.capacity,
                nl.col, reinterpret_cast<char4 *>(nl.shift), status);
        note_launches(5);
    } else {
        exclusive_scan(w.counts, nl.row_ptr, 0, w.scan_tmp, st);
        k_nl_total<<<1, 1, 0, st>>>(nl.row_ptr, nl.capacity, nl.n_pairs, status);
        note_launches(1);
    }
    return cudaPeekAtLastError() == cudaSuccess ? GM_OK : GM_ERR_CUDA;
}

}  // namespace gm
