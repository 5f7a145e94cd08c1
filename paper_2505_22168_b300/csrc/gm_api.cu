// gm_api.cu -- the extern "C" entry points of libgm (declared in include/gm.h).
//
// Energy + forces pipeline (one stream, no host synchronisation, no allocation):
//   moments (pair kernel)  -> psi [N][100]
//   contraction forward    -> G [Mp][384]
//   L1 GEMM  G W1          -> A1, D1          (phi, phi' of the first hidden layer)
//   L2 GEMM  A1 W2         -> dZ2, partial output sums (energies)
//   B1 GEMM  dZ2 W2^T      -> dZ1
//   B0 GEMM  dZ1 W1^T      -> dG [Mp][384]
//     (mixed path: the four layers may run as one kernel per tile or per cluster, mlp_form)
//   contraction backward   -> dpsi [N][100]
//   forces (pair kernel)   -> F [N][3], per-atom virial
//   per-structure FP64 reduction -> E [B], W [B][9]  (without the virial, the mixed path sums
//                             the energies inside the B1 GEMM or the cluster kernel)
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "gm_contract.h"
#include "gm_ensemble.h"
#include "gm_gemm.h"
#include "gm_internal.h"
#include "gm_md.h"
#include "gm_pair.h"
#include "gm_pgrad.h"
#include "gm_reduce.h"

using namespace gm;

static thread_local std::string g_last_error;

static gm_status fail(gm_status s, const char *msg) {
    g_last_error = msg;
    return s;
}

// ------------------------------------------------------------------ tracing
namespace gm {
static std::atomic<int64_t> g_launches{0};
static std::atomic<bool> g_prof{false};
static std::mutex g_prof_mu;
struct PendingStage {
    int stage;
    cudaEvent_t a, b;
};
static std::vector<PendingStage> g_pending;
static std::vector<PendingStage> g_graph_stages;  // event-record nodes of captured graphs
static std::vector<cudaEvent_t> g_event_pool;
static double g_stage_ms[N_STAGES];
static int64_t g_stage_cnt[N_STAGES];

static cudaEvent_t pool_event() {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void note_launches(int n) { g_launches += n; }

// While a stream is being captured into a CUDA graph the events become external
// event-record nodes: every replay records them again, and gm_profile_collect reads them
// after each replay (the caller synchronises first).
StageScope::StageScope(int s, cudaStream_t stream) : stage(s), st(stream), ev0(nullptr), in_graph(false) {
    if (!g_prof) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    in_graph = cs == cudaStreamCaptureStatusActive;
    cudaEvent_t e = nullptr;
    if (in_graph) cudaEventCreate(&e);
    else e = pool_event();
    if (in_graph) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else cudaEventRecord(e, st);
    ev0 = e;
}

StageScope::~StageScope() {
    if (!ev0) return;
    cudaEvent_t e = nullptr;
    if (in_graph) {
        cudaEventCreate(&e);
        cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    } else {
        e = pool_event();
        cudaEventRecord(e, st);
    }
    std::lock_guard<std::mutex> lk(g_prof_mu);
    (in_graph ? g_graph_stages : g_pending).push_back({stage, static_cast<cudaEvent_t>(ev0), e});
}
}  // namespace gm

struct gm_model {
    gm_model_desc d;
    int S, H, E;           // species, hidden width, shallow-ensemble heads (1 = plain model)
    int64_t n_param;
    RadialConst rc;
    int pair_tpa;          // lanes per atom in the pair kernels (0 = automatic)
    int forces_tpa;        // lanes per atom of the force kernel alone (0 = as pair_tpa / by size)
    char *buf;             // one device allocation holding everything below
    size_t buf_bytes;
    float *beta;           // [S][S][5][7] * n_basis^{-1/2}
    float *W1t;            // [H][384]  forward  (B[n=h][k=f])
    float *W1p;            // [384][H]  backward (B[n=f][k=h])
    float *W2t;            // [H][H]    forward  (B[n][k] = W2[k][n])
    float *W2;             // [H][H]    backward (B[n][k] = W2[n][k])
    __nv_bfloat16 *W1t_h, *W1p_h, *W2t_h, *W2_h;   // BF16 hi/lo pairs, rows [hi(K) | lo(K)]
    __half *W1p_f, *W2_f;  // FP16 copies of the backward weights, rows [fp16(K) | 0]
    int split_mask;        // GEMMs run with three hi/lo passes: 1 L1, 2 L2, 4 B1, 8 B0
    int f16_backward;      // backward GEMMs B1, B0 on FP16 operands in one pass (else split BF16)
    int fused_mlp;         // mixed path: the four network GEMMs as one kernel (where it applies)
    int mlp_cluster;       // CTAs per tile of the fused network kernel (0 by size, 1 one, 2/4/8)
    int mlp_ctas;          // CTAs of the persistent per-tile kernel (0: one per SM)
    int pg_split_mask;     // the same for the four network GEMMs of the parameter gradient
    int gemm_bn;           // tensor-core tile width (0 = by size)
    int gemm_cps;          // tensor-core GEMM blocks per SM (0 = by tile count)
    int debug_stall;       // GM_TUNE_DEBUG_STALL (failure-reporting tests)
    NlTuning nl;           // neighbour build launch shape
    float *b1, *b2, *w3, *b3, *sigma, *mu;
    float *w3e, *b3e;      // ensemble heads: w3e [E][H] (member-major), b3e [E]; w3 and b3 hold
                           // their mean (the head whose gradient is the mean force)
};

namespace {

struct Layout {
    size_t beta, W1t, W1p, W2t, W2, W1t_h, W1p_h, W2t_h, W2_h, W1p_f, W2_f, b1, b2, w3, b3, sigma, mu, w3e, b3e, total;
};

Layout model_layout(int S, int H, int E) {
    Layout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t start = (off + 255) & ~size_t(255);
        off = start + bytes;
        return start;
    };
    L.beta = take(sizeof(float) * S * S * NR * NB);
    L.W1t = take(sizeof(float) * H * NFP);
    L.W1p = take(sizeof(float) * NFP * H);
    L.W2t = take(sizeof(float) * H * H);
    L.W2 = take(sizeof(float) * H * H);
    L.W1t_h = take(4 * (size_t)H * NFP);
    L.W1p_h = take(4 * (size_t)NFP * H);
    L.W2t_h = take(4 * (size_t)H * H);
    L.W2_h = take(4 * (size_t)H * H);
    L.W1p_f = take(4 * (size_t)NFP * H);
    L.W2_f = take(4 * (size_t)H * H);
    L.b1 = take(sizeof(float) * H);
    L.b2 = take(sizeof(float) * H);
    L.w3 = take(sizeof(float) * H);
    L.b3 = take(sizeof(float) * 4);
    L.sigma = take(sizeof(float) * S);
    L.mu = take(sizeof(float) * S);
    L.w3e = take(sizeof(float) * (size_t)E * H);
    L.b3e = take(sizeof(float) * E);
    L.total = off;
    return L;
}

struct ThetaOff {
    int64_t beta, W1, b1, W2, b2, w3, b3, sigma, mu, total;
};

// flat theta: ..., w3 [H][E], b3 [E], sigma, mu (E = 1: w3 [H], b3 [1])
ThetaOff theta_offsets(int S, int H, int E = 1) {
    ThetaOff o;
    o.beta = 0;
    o.W1 = o.beta + (int64_t)S * S * NR * NB;
    o.b1 = o.W1 + (int64_t)NF * H;
    o.W2 = o.b1 + H;
    o.b2 = o.W2 + (int64_t)H * H;
    o.w3 = o.b2 + H;
    o.b3 = o.w3 + (int64_t)H * E;
    o.sigma = o.b3 + E;
    o.mu = o.sigma + S;
    o.total = o.mu + S;
    return o;
}

// FP16 weight copy in the hi slot of the same [rows][2K] layout (the lo slot stays zero).
__device__ __forceinline__ void put_f16(__half *dst, int K, int r, int k, float v) {
    dst[(size_t)r * 2 * K + k] = __float2half_rn(v);
}

// BF16 weight copy as a hi/lo pair: row r of a [rows][K] matrix becomes [hi(K) | lo(K)].
__device__ __forceinline__ void put_split(__nv_bfloat16 *dst, int K, int r, int k, float v) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    dst[(size_t)r * 2 * K + k] = hi;
    dst[(size_t)r * 2 * K + K + k] = __float2bfloat16_rn(v - __bfloat162float(hi));
}

__global__ void k_repack(const float *__restrict__ th, ThetaOff o, int S, int H, int E, float beta_scale, gm_model m) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t nbeta = (int64_t)S * S * NR * NB;
    for (int64_t q = tid; q < nbeta; q += stride) m.beta[q] = th[o.beta + q] * beta_scale;
    for (int64_t q = tid; q < (int64_t)H * NFP; q += stride) {
        // W1t[h][f] and W1p[f][h] for f < 384
        const int h = (int)(q / NFP), f = (int)(q % NFP);
        const float v = f < NF ? th[o.W1 + (int64_t)f * H + h] : 0.0f;
        m.W1t[q] = v;
        put_split(m.W1t_h, NFP, h, f, v);
        const int64_t qp = (int64_t)f * H + h;
        m.W1p[qp] = v;
        put_split(m.W1p_h, H, f, h, v);
        put_f16(m.W1p_f, H, f, h, v);
    }
    for (int64_t q = tid; q < (int64_t)H * H; q += stride) {
        const int r = (int)(q / H), c = (int)(q % H);
        const float v = th[o.W2 + q];  // W2[r][c]
        m.W2[q] = v;
        put_split(m.W2_h, H, r, c, v);
        put_f16(m.W2_f, H, r, c, v);
        const int64_t qt = (int64_t)c * H + r;  // W2t[c][r] = W2[r][c]
        m.W2t[qt] = v;
        put_split(m.W2t_h, H, c, r, v);
    }
    for (int64_t q = tid; q < H; q += stride) {
        m.b1[q] = th[o.b1 + q];
        m.b2[q] = th[o.b2 + q];
        float sw = 0.0f;
        for (int e = 0; e < E; ++e) {
            const float w = th[o.w3 + q * E + e];
            m.w3e[(int64_t)e * H + q] = w;
            sw += w;
        }
        m.w3[q] = sw / (float)E;
    }
    for (int64_t q = tid; q < S; q += stride) {
        m.sigma[q] = th[o.sigma + q];
        m.mu[q] = th[o.mu + q];
    }
    if (tid == 0) {
        float sb = 0.0f;
        for (int e = 0; e < E; ++e) {
            m.b3e[e] = th[o.b3 + e];
            sb += th[o.b3 + e];
        }
        m.b3[0] = sb / (float)E;
    }
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

struct EfWs {
    float *psi, *dpsi, *G, *A1, *D1, *dZ2, *dZ1, *dG, *nn_part, *vir_atom;
    unsigned long long *red_acc;   // fixed-point structure sums (cleared by the position split)
    int n_red_acc;
    float4 *pos_hi, *pos_lo;   // hi/lo FP32 split of the positions (pair displacements)
    // shallow ensembles (E > 1): per-head partial sums, head-energy accumulators, per-head forces,
    // and for the Jacobian mode the dE/dG and dE/dPsi of a chunk of heads (ens_head_chunk)
    float *nn_ens, *Fk, *dZ2h, *dZ1h, *dGh, *dpsih;
    unsigned long long *ens_acc;
};

// Heads whose backward contraction and force pass share one launch in the Jacobian mode: as
// many as keep the chunk within 16,384 virtual atoms (small systems, where one head's pass
// leaves most of the GPU idle), one at a time above
int ens_head_chunk(int E, int N) {
    const int hc = N > 0 ? 16384 / N : E;
    return hc < 1 ? 1 : (hc > E ? E : hc);
}

EfWs carve_ef(Carve &c, int B, int N, int H, int E = 1) {
    EfWs w;
    const int Mp = round_up(N, TILE_M);
    const size_t n1 = N > 0 ? (size_t)N : 1, m1 = Mp > 0 ? (size_t)Mp : 1;
    w.psi = c.take<float>(n1 * NPSI);
    w.dpsi = c.take<float>(n1 * NPSI);
    w.pos_hi = c.take<float4>(n1);
    w.pos_lo = c.take<float4>(n1);
    w.G = c.take<float>(m1 * NFP);
    w.A1 = c.take<float>(m1 * H);
    w.D1 = c.take<float>(m1 * H);
    w.dZ2 = c.take<float>(m1 * H);
    w.dZ1 = c.take<float>(m1 * H);
    w.dG = c.take<float>(m1 * NFP);
    w.nn_part = c.take<float>(m1 * (H / 32));
    w.vir_atom = c.take<float>(n1 * 9);
    // the structure sums and, for an ensemble, the head-energy sums right after them: the
    // position-split kernel clears both
    const size_t n_acc = reduce_acc_words(B) + (E > 1 ? ens_acc_words(B, E) : 0);
    w.red_acc = c.take<unsigned long long>(n_acc);
    w.n_red_acc = (int)n_acc;
    w.nn_ens = w.Fk = w.dZ2h = w.dZ1h = w.dGh = w.dpsih = nullptr;
    w.ens_acc = nullptr;
    if (E > 1) {
        w.nn_ens = c.take<float>(m1 * E * (H / 32));
        w.Fk = c.take<float>((size_t)E * n1 * 3);
        w.ens_acc = w.red_acc ? w.red_acc + reduce_acc_words(B) : nullptr;
        const int hc = ens_head_chunk(E, N);
        w.dZ2h = hc > 1 ? c.take<float>((size_t)hc * m1 * H) : w.dZ2;
        w.dZ1h = hc > 1 ? c.take<float>((size_t)hc * m1 * H) : w.dZ1;
        w.dGh = hc > 1 ? c.take<float>((size_t)hc * m1 * NFP) : w.dG;
        w.dpsih = hc > 1 ? c.take<float>((size_t)hc * n1 * NPSI) : w.dpsi;
    }
    return w;
}

size_t ef_workspace_bytes(int B, int N, int H, int E) {
    Carve c(reinterpret_cast<void *>(256), ~size_t(0) >> 1);
    carve_ef(c, B, N, H, E);
    return c.off + 256;
}

// MD: the neighbour build's workspace (with the search slab for the list's capacity), the
// energy/force workspace, and the integrator's words (skin flag, kinetic-energy accumulators,
// per-structure thermostat velocity factors)
struct MdWs {
    void *nl;
    size_t nl_bytes;
    EfWs ef;
    int32_t *flag;
    unsigned long long *acc;
    double *pending;
};

MdWs carve_md(Carve &c, int B, int N, int H, int64_t cap) {
    MdWs w;
    w.nl_bytes = nl_workspace_bytes(B, N, cap);
    w.nl = c.take<char>(w.nl_bytes);
    w.ef = carve_ef(c, B, N, H);
    w.flag = c.take<int32_t>(64);
    w.acc = c.take<unsigned long long>(reduce_acc_words(B));
    w.pending = c.take<double>(B);
    return w;
}

size_t md_workspace_bytes(int B, int N, int H, int64_t cap) {
    Carve c(reinterpret_cast<void *>(256), ~size_t(0) >> 1);
    carve_md(c, B, N, H, cap);
    return c.off + 256;
}

struct PgWs {
    float *psi, *psid, *psib, *psidb, *GG, *Gbs, *Z, *A1s, *P1, *Q1, *Zd1, *Zb2s, *Zb1s, *Y3, *t_sig, *t_c, *t_cs,
        *beta_part, *wg_part;
    float4 *pos_hi, *pos_lo;
    __nv_bfloat16 *hl;   // mixed path: hi/lo BF16 copy of the current GEMM's A operand [2 Mp][2 K]
};

PgWs carve_pg(Carve &c, int N, int H, int S) {
    PgWs w;
    const int Mp = round_up(N, TILE_M);
    const size_t n1 = N > 0 ? (size_t)N : 1, m1 = Mp > 0 ? (size_t)Mp : 1;
    w.psi = c.take<float>(n1 * NPSI);
    w.psid = c.take<float>(n1 * NPSI);
    w.pos_hi = c.take<float4>(n1);
    w.pos_lo = c.take<float4>(n1);
    w.psib = c.take<float>(n1 * NPSI);
    w.psidb = c.take<float>(n1 * NPSI);
    w.GG = c.take<float>(2 * m1 * NFP);
    w.Gbs = c.take<float>(2 * m1 * NFP);
    w.Z = c.take<float>(2 * m1 * H);
    w.A1s = c.take<float>(2 * m1 * H);
    w.P1 = c.take<float>(m1 * H);
    w.Q1 = c.take<float>(m1 * H);
    w.Zd1 = c.take<float>(m1 * H);
    w.Zb2s = c.take<float>(2 * m1 * H);
    w.Zb1s = c.take<float>(2 * m1 * H);
    w.Y3 = c.take<float>(m1 * H);
    w.t_sig = c.take<float>(m1);
    w.t_c = c.take<float>(m1);
    w.t_cs = c.take<float>(m1);
    w.beta_part = c.take<float>((size_t)(pg_beta_blocks(N, S) + 1) * S * S * NR * NB);
    w.hl = c.take<__nv_bfloat16>(2 * m1 * 2 * (size_t)(H > NFP ? H : NFP));
    size_t scratch = std::max((size_t)wgrad_ksplit(2 * Mp, NFP, H) * NFP * H,         // weight-gradient slices
                              (size_t)wgrad_ksplit(2 * Mp, H, H) * H * H);            // (W1, then W2),
    scratch = std::max(scratch, colsum_part_floats(Mp, H));                           // later column sums
    scratch = std::max(scratch, pg_tail_part_floats(N, S));                           // and species sums
    w.wg_part = c.take<float>(scratch);
    return w;
}

size_t pg_workspace_bytes(int N, int H, int S) {
    Carve c(reinterpret_cast<void *>(256), ~size_t(0) >> 1);
    carve_pg(c, N, H, S);
    return c.off + 256;
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

// Argument checks shared by every entry point that takes a system and a neighbour list
// (declared in gm_internal.h): every pointer the kernels dereference is non-null where
// needed and aligned for its element type, so a bad pointer is rejected on the host.
namespace gm {

gm_status check_system(const gm_model *m, const gm_system *s) {
    if (!m || !s) return fail(GM_ERR_ARG, "null model or system");
    if (s->n_structures < 1 || s->n_atoms < 0) return fail(GM_ERR_ARG, "n_structures must be >= 1 and n_atoms >= 0");
    if (s->n_atoms > GM_MAX_ATOMS) return fail(GM_ERR_UNSUPPORTED, "more than GM_MAX_ATOMS atoms");
    if (!s->atom_ptr || !s->cell || !s->pbc) return fail(GM_ERR_ARG, "atom_ptr, cell and pbc must be non-null");
    if (s->n_atoms > 0 && (!s->pos || !s->species)) return fail(GM_ERR_ARG, "pos and species must be non-null");
    if (!aligned(s->pos, 8) || !aligned(s->cell, 8) || !aligned(s->atom_ptr, 4) || !aligned(s->species, 4))
        return fail(GM_ERR_ARG, "misaligned system pointer");
    return GM_OK;
}

gm_status check_nlist(const gm_system *s, const gm_nlist *nl, bool need_pairs) {
    if (!nl || !nl->row_ptr || !nl->n_pairs) return fail(GM_ERR_ARG, "null neighbour list field");
    if (nl->capacity < 0) return fail(GM_ERR_ARG, "negative capacity");
    if (nl->capacity > 0 && (!nl->col || !nl->shift)) return fail(GM_ERR_ARG, "null col/shift with capacity > 0");
    if (!aligned(nl->shift, 4) || !aligned(nl->col, 4) || !aligned(nl->row_ptr, 4))
        return fail(GM_ERR_ARG, "misaligned neighbour list pointer");
    (void)s;
    (void)need_pairs;
    return GM_OK;
}

gm_status launch_status() {
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) return fail(GM_ERR_CUDA, cudaGetErrorString(e));
    return GM_OK;
}

gm_status check_stream_device(cudaStream_t stream) {
    int cur = -1, sdev = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return fail(GM_ERR_CUDA, "cudaGetDevice failed");
    if (cudaStreamGetDevice(stream, &sdev) != cudaSuccess) return fail(GM_ERR_ARG, "invalid stream");
    if (sdev != cur) return fail(GM_ERR_ARG, "the stream belongs to another device than the current one");
    return GM_OK;
}

}  // namespace gm

namespace {

PairArgs pair_args(const gm_model *m, const gm_system *s, const gm_nlist *nl, const float4 *pos_hi,
                   const float4 *pos_lo, int32_t *status) {
    PairArgs a;
    a.N = s->n_atoms;
    a.B = s->n_structures;
    a.S = m->S;
    a.atom_ptr = s->atom_ptr;
    a.pos = s->pos;
    a.pos_hi = pos_hi;
    a.pos_lo = pos_lo;
    a.species = s->species;
    a.cell = s->cell;
    a.row_ptr = nl->row_ptr;
    a.col = nl->col;
    a.shift = reinterpret_cast<const char4 *>(nl->shift);
    a.beta = m->beta;
    a.rc = m->rc;
    a.status = status;
    return a;
}

// Lanes per atom of the moments kernel, measured on B300 over Li3PO4-like crystals of 4k-131k
// atoms, the 256-box batch, the 1536-atom EMIM box and the 7920-atom training batch: the
// reduce-scatter kernel's 128-thread blocks below 12k atoms (8 at 4096, 32 at 8192), then the
// component-split kernel (two lanes of a pair keep 50 sums each, two blocks per SM) with 4
// lanes per atom, and with 2 from ~25k (131,072 atoms 320 -> 265 us, the batch 112 -> 101 us
// against one lane per atom)
int choose_tpa(const gm_model *m, int N) {
    if (m->pair_tpa > 0) return m->pair_tpa;
    if (N >= 24576) return 2;
    if (N >= 12288) return 4;
    if (N >= 6144) return 32;
    if (N >= 3072) return 8;
    return 32;
}

// Lanes per atom of the tangent moments (parameter gradient): at most 4, as the kernel sums
// its 100 accumulators over the lanes with a plain all-reduce (8 lanes took 101 us against
// 57 us for 4 at 7920 atoms); one lane per atom from ~49k atoms
int choose_tangent_tpa(const gm_model *m, int N) {
    if (m->pair_tpa > 0) return std::min(m->pair_tpa, 4);
    return N >= 49152 ? 1 : 4;
}

// Lanes per atom of the force kernel: with four or more lanes an atom's dE/dPsi sits once in
// shared memory (106 registers without the virial, four 128-thread blocks per SM); 32 below
// 3072 atoms, 8 below 49,152, 4 above (131,072 atoms 342 -> 326 us, the 256-box batch 149 ->
// 133 us against 8; 8 faster from 4k to 8k and at 24k, even at 12k-16k)
int choose_forces_tpa(const gm_model *m, int N) {
    if (m->forces_tpa > 0) return m->forces_tpa;
    if (m->pair_tpa > 0) return m->pair_tpa;
    return N >= 49152 ? 4 : (N >= 3072 ? 8 : 32);
}


}  // namespace

namespace gm {
const gm_model_desc *model_desc(const gm_model *m) { return &m->d; }
const NlTuning &nl_tuning(const gm_model *m) { return m->nl; }
gm_status set_last_error(gm_status s, const char *msg) { return fail(s, msg); }
}  // namespace gm

extern "C" {

int64_t gm_param_count(const gm_model_desc *d) {
    if (!d || d->n_species < 1 || d->n_hidden < 1) return -1;
    return theta_offsets(d->n_species, d->n_hidden, d->n_ensemble > 1 ? d->n_ensemble : 1).total;
}

gm_status gm_model_create(const gm_model_desc *d, gm_model **out) {
    if (!d || !out) return fail(GM_ERR_ARG, "null argument");
    *out = nullptr;
    if (d->n_species < 1 || d->n_species > MAX_S) return fail(GM_ERR_UNSUPPORTED, "n_species must be in 1..16");
    if (d->n_basis != NB || d->n_radial != NR) return fail(GM_ERR_UNSUPPORTED, "n_basis must be 7 and n_radial 5");
    if (d->n_hidden < 64 || d->n_hidden > 512 || d->n_hidden % 64 != 0)
        return fail(GM_ERR_UNSUPPORTED, "n_hidden must be a multiple of 64 in 64..512");
    if (d->activation != GM_ACT_TANH && d->activation != GM_ACT_SILU) return fail(GM_ERR_ARG, "bad activation");
    if (d->precision != GM_PREC_FP32 && d->precision != GM_PREC_MIXED) return fail(GM_ERR_ARG, "bad precision");
    if (!(d->r_cut > 0.0) || !(d->r_min >= 0.0) || !(d->r_min < d->r_cut)) return fail(GM_ERR_ARG, "bad radii");
    if (d->basis != GM_BASIS_GAUSSIAN && d->basis != GM_BASIS_BESSEL) return fail(GM_ERR_ARG, "bad basis");
    if (d->n_ensemble < 0 || d->n_ensemble > GM_MAX_ENSEMBLE) return fail(GM_ERR_UNSUPPORTED, "n_ensemble must be in 0..32");
    gm_model *m = new gm_model();
    m->d = *d;
    m->S = d->n_species;
    m->H = d->n_hidden;
    m->E = d->n_ensemble > 1 ? d->n_ensemble : 1;
    m->n_param = theta_offsets(m->S, m->H, m->E).total;
    m->rc.r_cut = (float)d->r_cut;
    m->rc.inv_r_cut = (float)(1.0 / d->r_cut);
    m->rc.pi_inv_r_cut = (float)(3.14159265358979323846 / d->r_cut);
    m->rc.gamma = (float)((double)(NB * NB) / (d->r_cut * d->r_cut));
    m->rc.gamma_l2 = (float)((double)(NB * NB) / (d->r_cut * d->r_cut) * 1.44269504088896340736);
    for (int k = 0; k < NB; ++k) m->rc.mu[k] = (float)(d->r_min + k * (d->r_cut - d->r_min) / (NB - 1));
    m->rc.basis = d->basis;
    for (int k = 0; k < NB; ++k) {
        const double n1 = k + 1.0, n2 = k + 2.0;
        m->rc.bes_a[k] = (float)(((k & 1) ? -1.0 : 1.0) * sqrt(2.0) * 3.14159265358979323846 / pow(d->r_cut, 1.5) *
                                 n1 * n2 / sqrt(n1 * n1 + n2 * n2));
    }
    m->pair_tpa = 0;
    m->forces_tpa = 0;
    m->split_mask = 12;
    m->f16_backward = 1;
    m->fused_mlp = 2;
    m->mlp_cluster = 0;
    m->mlp_ctas = 0;
    m->pg_split_mask = 15;
    m->gemm_bn = 0;
    m->gemm_cps = 0;
    m->debug_stall = 0;
    m->nl = NlTuning();
    Layout L = model_layout(m->S, m->H, m->E);
    m->buf_bytes = L.total;
    if (cudaMalloc(&m->buf, L.total) != cudaSuccess) {
        delete m;
        return fail(GM_ERR_CUDA, "cudaMalloc of model weights failed");
    }
    cudaMemset(m->buf, 0, L.total);
    m->beta = reinterpret_cast<float *>(m->buf + L.beta);
    m->W1t = reinterpret_cast<float *>(m->buf + L.W1t);
    m->W1p = reinterpret_cast<float *>(m->buf + L.W1p);
    m->W2t = reinterpret_cast<float *>(m->buf + L.W2t);
    m->W2 = reinterpret_cast<float *>(m->buf + L.W2);
    m->W1t_h = reinterpret_cast<__nv_bfloat16 *>(m->buf + L.W1t_h);
    m->W1p_h = reinterpret_cast<__nv_bfloat16 *>(m->buf + L.W1p_h);
    m->W2t_h = reinterpret_cast<__nv_bfloat16 *>(m->buf + L.W2t_h);
    m->W2_h = reinterpret_cast<__nv_bfloat16 *>(m->buf + L.W2_h);
    m->W1p_f = reinterpret_cast<__half *>(m->buf + L.W1p_f);
    m->W2_f = reinterpret_cast<__half *>(m->buf + L.W2_f);
    m->b1 = reinterpret_cast<float *>(m->buf + L.b1);
    m->b2 = reinterpret_cast<float *>(m->buf + L.b2);
    m->w3 = reinterpret_cast<float *>(m->buf + L.w3);
    m->b3 = reinterpret_cast<float *>(m->buf + L.b3);
    m->sigma = reinterpret_cast<float *>(m->buf + L.sigma);
    m->mu = reinterpret_cast<float *>(m->buf + L.mu);
    m->w3e = reinterpret_cast<float *>(m->buf + L.w3e);
    m->b3e = reinterpret_cast<float *>(m->buf + L.b3e);
    *out = m;
    return GM_OK;
}

gm_status gm_model_set_params(gm_model *m, const float *theta, struct CUstream_st *stream) {
    if (!m || !theta) return fail(GM_ERR_ARG, "null argument");
    if (!aligned(theta, 4)) return fail(GM_ERR_ARG, "misaligned theta");
    ThetaOff o = theta_offsets(m->S, m->H, m->E);
    const float scale = (float)(1.0 / sqrt((double)NB));
    k_repack<<<296, 256, 0, stream>>>(theta, o, m->S, m->H, m->E, scale, *m);
    note_launches(1);
    return launch_status();
}

size_t gm_model_device_bytes(const gm_model *m) { return m ? m->buf_bytes : 0; }

int32_t gm_model_pair_lanes(const gm_model *m, int32_t n_atoms) {
    if (!m || n_atoms < 0) return -1;
    return choose_tpa(m, n_atoms);
}

int32_t gm_model_force_lanes(const gm_model *m, int32_t n_atoms) {
    if (!m || n_atoms < 0) return -1;
    return choose_forces_tpa(m, n_atoms);
}

gm_status gm_model_set_tuning(gm_model *m, int32_t key, int32_t value) {
    if (!m) return fail(GM_ERR_ARG, "null model");
    switch (key) {
    case GM_TUNE_PAIR_TPA:
        if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8 && value != 16 && value != 32)
            return fail(GM_ERR_ARG, "pair TPA must be 0, 1, 2, 4, 8, 16 or 32");
        m->pair_tpa = value;
        return GM_OK;
    case GM_TUNE_FORCES_TPA:
        if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8 && value != 16 && value != 32)
            return fail(GM_ERR_ARG, "force TPA must be 0, 1, 2, 4, 8, 16 or 32");
        m->forces_tpa = value;
        return GM_OK;
    case GM_TUNE_SPLIT_MASK:
        if (value < 0 || value > 15) return fail(GM_ERR_ARG, "split mask must be in 0..15");
        m->split_mask = value;
        return GM_OK;
    case GM_TUNE_PG_SPLIT_MASK:
        if (value < 0 || value > 15) return fail(GM_ERR_ARG, "split mask must be in 0..15");
        m->pg_split_mask = value;
        return GM_OK;
    case GM_TUNE_FUSED_MLP:
        if (value < 0 || value > 2) return fail(GM_ERR_ARG, "fused network mode must be 0, 1 or 2");
        m->fused_mlp = value;
        return GM_OK;
    case GM_TUNE_MLP_CLUSTER:
        if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8)
            return fail(GM_ERR_ARG, "network cluster size must be 0, 1, 2, 4 or 8");
        m->mlp_cluster = value;
        return GM_OK;
    case GM_TUNE_MLP_CTAS:
        if (value < 0 || value > 4096) return fail(GM_ERR_ARG, "fused network CTAs must be in 0..4096");
        m->mlp_ctas = value;
        return GM_OK;
    case GM_TUNE_F16_BACKWARD:
        if (value != 0 && value != 1) return fail(GM_ERR_ARG, "FP16 backward flag must be 0 or 1");
        m->f16_backward = value;
        return GM_OK;
    case GM_TUNE_DEBUG_STALL:
        if (value < 0 || value > 2) return fail(GM_ERR_ARG, "debug stall must be 0, 1 or 2");
        m->debug_stall = value;
        m->nl.debug_stall = value == 1 ? 1 : 0;
        return GM_OK;
    case GM_TUNE_GEMM_BN:
        if (value != 0 && value != 64 && value != 128 && value != 256) return fail(GM_ERR_ARG, "bad GEMM tile width");
        m->gemm_bn = value;
        return GM_OK;
    case GM_TUNE_GEMM_CPS:
        if (value < 0 || value > 2) return fail(GM_ERR_ARG, "GEMM blocks per SM must be 0, 1 or 2");
        m->gemm_cps = value;
        return GM_OK;
    case GM_TUNE_NL_MODE:
        if (value != GM_NL_MODE_AUTO && value != GM_NL_MODE_PHASES) return fail(GM_ERR_ARG, "bad neighbour mode");
        m->nl.mode = value;
        return GM_OK;
    case GM_TUNE_NL_SPLIT:
        if (value < 0 || value > 16) return fail(GM_ERR_ARG, "neighbour split must be in 0..16");
        m->nl.split = value;
        return GM_OK;
    case GM_TUNE_NL_BLOCKS:
        if (value < 0 || value > 4096) return fail(GM_ERR_ARG, "neighbour blocks must be in 0..4096");
        m->nl.blocks = value;
        return GM_OK;
    case GM_TUNE_NL_ITEMS:
        if (value < 0 || value > 3) return fail(GM_ERR_ARG, "neighbour item mode must be 0, 1, 2 or 3");
        m->nl.items = value;
        return GM_OK;
    case GM_TUNE_NL_TWO_PASS:
        if (value != 0 && value != 1) return fail(GM_ERR_ARG, "neighbour two-pass flag must be 0 or 1");
        m->nl.two_pass = value;
        return GM_OK;
    }
    return fail(GM_ERR_ARG, "unknown tuning key");
}

void gm_model_destroy(gm_model *m) {
    if (!m) return;
    cudaFree(m->buf);
    delete m;
}

gm_status gm_workspace_size(const gm_model *m, int32_t n_structures, int32_t n_atoms, int64_t nl_capacity,
                            int32_t op, size_t *bytes) {
    if (!m || !bytes || n_structures < 1 || n_atoms < 0 || nl_capacity < 0) return fail(GM_ERR_ARG, "bad argument");
    switch (op) {
    case GM_OP_NEIGHBORS: *bytes = nl_workspace_bytes(n_structures, n_atoms, nl_capacity); return GM_OK;
    case GM_OP_ENERGY_FORCES: *bytes = ef_workspace_bytes(n_structures, n_atoms, m->H, m->E); return GM_OK;
    case GM_OP_PARAM_GRAD: *bytes = pg_workspace_bytes(n_atoms, m->H, m->S); return GM_OK;
    case GM_OP_MD: *bytes = md_workspace_bytes(n_structures, n_atoms, m->H, nl_capacity); return GM_OK;
    default: return fail(GM_ERR_ARG, "unknown op");
    }
}

gm_status gm_build_neighbors(const gm_model *m, const gm_system *sys, gm_nlist *nl, void *ws, size_t ws_bytes,
                             int32_t *status, struct CUstream_st *stream) {
    gm_status s = check_system(m, sys);
    if (s != GM_OK) return s;
    if ((s = check_nlist(sys, nl, false)) != GM_OK) return s;
    if (!status) return fail(GM_ERR_ARG, "null status");
    if (ws_bytes < nl_workspace_min_bytes(sys->n_structures, sys->n_atoms))
        return fail(GM_ERR_WORKSPACE, "workspace too small");
    {
        StageScope sc(ST_NEIGHBORS, stream);
        s = nl_build(*sys, m->d.r_cut, m->S, *nl, ws, ws_bytes, status, stream, m->nl);
    }
    if (s != GM_OK) return fail(s, "neighbour build launch failed");
    return launch_status();
}

// forces_to_clear (the step's force output) and, with it, the structure-sum accumulators are
// cleared by the position-split kernel
static gm_status forward_to_features(const gm_model *m, const gm_system *sys, const gm_nlist *nl, EfWs &w,
                                     float *psi_out, float *features_out, float *forces_to_clear, int32_t *status,
                                     cudaStream_t st) {
    const int N = sys->n_atoms;
    const int Mp = round_up(N, TILE_M);
    PairArgs a = pair_args(m, sys, nl, w.pos_hi, w.pos_lo, status);
    float *psi = psi_out ? psi_out : w.psi;
    {
        StageScope sc(ST_MOMENTS, st);
        launch_split_pos(N, sys->pos, sys->species, w.pos_hi, w.pos_lo, forces_to_clear,
                         forces_to_clear ? w.red_acc : nullptr, w.n_red_acc, st);
        launch_moments(a, choose_tpa(m, N), psi, st);
    }
    {
        StageScope sc(ST_CONTRACT_FWD, st);
        if (m->d.precision == GM_PREC_MIXED && features_out == nullptr)
            launch_contract_fwd_bf16(psi, N, Mp, reinterpret_cast<__nv_bfloat16 *>(w.G), nullptr,
                                     (m->split_mask & 1) != 0, st);
        else
            launch_contract_fwd_f32(psi, N, Mp, w.G, features_out, st);
    }
    w.psi = psi;
    return launch_status();
}

// The mixed path's network runs as one fused kernel when the model's width allows it, the
// backward GEMMs take FP16 and the forward ones single-pass BF16, and no ensemble partial sums
// or other output head are asked for.  Two forms:
//   per tile   one CTA per 128-atom tile runs the four layers one after another
//              (gm_mlp_fused.cuh); every CTA streams all the weights (1.8 MB at width 512)
//   cluster    each tile split over a cluster of 2, 4 or 8 CTAs along the hidden width, the
//              layer slices all-gathered between layers (gm_mlp_cluster.cuh); each CTA
//              streams 1/CS of the weights but receives (CS - 1)/CS of every gathered layer
// GM_TUNE_FUSED_MLP: 0 never (four GEMM launches), 1 always, 2 (default) by size;
// GM_TUNE_MLP_CLUSTER: 0 (default) cluster size by size, 1 per tile, 2, 4 or 8.
// By size (B300, whole energy/force step, width 512): below 16 tiles the four GEMM launches
// (1536 atoms: 89 us against 93-97 with a cluster); a cluster while all its CTAs fit on the
// GPU at once, at most 4 wide (4096 atoms: 141 us with 4 against 156 for the GEMMs; 5184
// atoms, width 256: 166 with 2 against 175; 8192 atoms: 215 with 2 against 233); one CTA per
// tile above that (16,384 atoms: 322 against 349).
// Returns MLP_GEMMS, MLP_TILE or MLP_CLUSTER (with the cluster size in *cs).
enum { MLP_GEMMS = 0, MLP_TILE = 1, MLP_CLUSTER = 2 };
static int mlp_form(const gm_model *m, bool ens, bool from_l2, const float *head, int n_atoms, int *cs) {
    *cs = 1;
    if (m->d.precision != GM_PREC_MIXED || m->fused_mlp == 0 || !m->f16_backward || !mlp_fused_supported(m->H) ||
        ens || from_l2 || head != nullptr || (m->split_mask & 3) != 0)
        return MLP_GEMMS;
    const int tiles = (n_atoms + TILE_M - 1) / TILE_M;
    if (m->mlp_cluster >= 2) {
        if (mlp_cluster_capacity(m->d.activation, m->H, m->mlp_cluster) <= 0) return MLP_GEMMS;
        *cs = m->mlp_cluster;
        return MLP_CLUSTER;
    }
    if (m->mlp_cluster == 0 && tiles >= 16) {
        for (int c = 4; c >= 2; c /= 2) {
            if (!mlp_cluster_supported(m->H, c) || tiles * c > 148) continue;
            if (tiles <= mlp_cluster_capacity(m->d.activation, m->H, c)) {
                *cs = c;
                return MLP_CLUSTER;
            }
        }
    }
    if (m->fused_mlp == 1 || tiles >= 16) return MLP_TILE;
    return MLP_GEMMS;
}

// The four network GEMMs: features -> energies (partial sums) and dE/dG.  energy (mixed
// path only): the structure energies are summed inside the B1 GEMM and written there.
//   head:      output-layer weights whose gradient is taken (null: the model's w3, which for
//              a shallow ensemble is the heads' mean)
//   ens:       also write every ensemble head's partial sums (w.nn_ens) in the L2 epilogue
//   from_l2:   skip L1 (its outputs A1, D1 are still in the workspace from an earlier pass)
//   nheads:    with from_l2 and head, the backward pass of nheads heads (weights head + u H):
//              one L2 GEMM whose epilogue writes every head's dZ2 rows (u Mp ..), then B1 and
//              B0 once over nheads Mp rows (phi'(z1) read at row mod Mp) into the stacked dZ1
//              and dG; no output-layer partial sums
static gm_status network_fwd_bwd(const gm_model *m, const gm_system *sys, EfWs &w, int Mp, int32_t *status,
                                 cudaStream_t st, double *energy = nullptr, const float *head = nullptr,
                                 bool ens = false, bool from_l2 = false, int nheads = 1) {
    const int H = m->H;
    const bool stacked = from_l2 && head != nullptr;   // the Jacobian mode's heads
    const int l2 = stacked ? EPI_L2H : (ens ? EPI_L2E : EPI_L2);
    EpiArgs e{};
    e.n_atoms = sys->n_atoms;
    e.n_species = m->S;
    e.species = sys->species;
    e.w3 = head ? head : m->w3;
    e.sigma = m->sigma;
    e.nn_part = w.nn_part;
    e.n_ens = ens ? m->E : 1;
    e.w3e = m->w3e;
    e.nn_ens = w.nn_ens;
    e.nn_ens_ld = (size_t)Mp;
    e.n_heads = nheads;
    int cs = 1;
    const int form = mlp_form(m, ens, from_l2, head, sys->n_atoms, &cs);
    if (form != MLP_GEMMS) {
        FusedMlpArgs fa;
        fa.n_atoms = sys->n_atoms;
        fa.n_species = m->S;
        fa.species = sys->species;
        fa.b1 = m->b1;
        fa.b2 = m->b2;
        fa.w3 = m->w3;
        fa.sigma = m->sigma;
        fa.D1 = reinterpret_cast<__half *>(w.D1);
        fa.nn_part = w.nn_part;
        fa.dG = w.dG;
        fa.debug_stall = m->debug_stall == 2 ? 1 : 0;
        fa.ctas = m->mlp_ctas;
        StageScope sc(ST_MLP_FUSED, st);
        gm_status s;
        if (form == MLP_CLUSTER) {
            fa.xa1 = reinterpret_cast<__nv_bfloat16 *>(w.A1);
            fa.xdz2 = reinterpret_cast<__nv_bfloat16 *>(w.dZ2);
            fa.xdz1 = reinterpret_cast<__nv_bfloat16 *>(w.dZ1);
            if (energy) {
                fa.atom_ptr = sys->atom_ptr;
                fa.n_structures = sys->n_structures;
                fa.mu = m->mu;
                fa.b3 = m->b3;
                fa.red_acc = w.red_acc;
                fa.energy = energy;
            }
            s = mlp_cluster(m->d.activation, Mp, H, cs, reinterpret_cast<const __nv_bfloat16 *>(w.G), m->W1t_h,
                            m->W2t_h, m->W2_f, m->W1p_f, fa, status, st);
        } else {
            s = mlp_fused(m->d.activation, Mp, H, reinterpret_cast<const __nv_bfloat16 *>(w.G), m->W1t_h, m->W2t_h,
                          m->W2_f, m->W1p_f, fa, status, st);
        }
        return s == GM_OK ? GM_OK : fail(s, "fused network kernel failed");
    }
    if (m->d.precision == GM_PREC_MIXED) {
        typedef __nv_bfloat16 bf;
        bf *G = reinterpret_cast<bf *>(w.G), *A1 = reinterpret_cast<bf *>(w.A1);
        float *D1 = w.D1;
        const int sp = m->split_mask;
        bf *dZ2 = reinterpret_cast<bf *>(w.dZ2), *dZ1 = reinterpret_cast<bf *>(w.dZ1);
        gm_status s;
        if (!from_l2) {
            e.bias = m->b1;
            e.out0 = A1;
            e.out1 = D1;
            e.lo_out = (sp & 2) != 0;   // lo halves only where the consuming GEMM runs split
            e.debug_stall = m->debug_stall == 2 ? 1 : 0;
            StageScope sc(ST_GEMM_L1, st);
            if ((s = gemm_bf16(EPI_L1, m->d.activation, G, m->W1t_h, Mp, H, NFP, (sp & 1) != 0, e, status, st, m->gemm_bn, m->gemm_cps)) != GM_OK)
                return fail(s, "tcgen05 GEMM L1 failed");
            e.debug_stall = 0;
        }
        // backward operands: FP16 in one pass (they are bounded: |dE/dz| <= |sigma w3| max phi'),
        // or BF16 hi/lo split as the split mask says
        const int f16 = m->f16_backward;
        const bf *W2b = f16 ? reinterpret_cast<const bf *>(m->W2_f) : m->W2_h;
        const bf *W1b = f16 ? reinterpret_cast<const bf *>(m->W1p_f) : m->W1p_h;
        e.bias = m->b2;
        e.out1 = nullptr;
        e.lo_out = f16 ? 0 : (sp & 4) != 0;
        e.out_f16 = f16;
        e.out0 = dZ2;
        e.head_stride = (size_t)Mp * 2 * H;                  // [Mp][2H] 16-bit rows per head
        {
            StageScope sc(ST_GEMM_L2, st);
            if ((s = gemm_bf16(l2, m->d.activation, A1, m->W2t_h, Mp, H, H, (sp & 2) != 0, e, status, st, m->gemm_bn, m->gemm_cps)) != GM_OK)
                return fail(s, "tcgen05 GEMM L2 failed");
        }
        e.out0 = dZ1;
        e.aux = D1;
        e.aux_rows = nheads > 1 ? Mp : 0;
        e.lo_out = f16 ? 0 : (sp & 8) != 0;
        if (energy) {
            e.atom_ptr = sys->atom_ptr;
            e.n_structures = sys->n_structures;
            e.mu = m->mu;
            e.b3 = m->b3;
            e.red_acc = w.red_acc;
            e.energy = energy;
        }
        {
            StageScope sc(ST_GEMM_B1, st);
            if ((s = gemm_bf16(EPI_B1, 0, dZ2, W2b, nheads * Mp, H, H, f16 ? 0 : (sp & 4) != 0, e, status, st,
                               m->gemm_bn, m->gemm_cps, f16)) != GM_OK)
                return fail(s, "tcgen05 GEMM B1 failed");
        }
        e.out0 = w.dG;
        e.energy = nullptr;
        e.out_f16 = 0;
        {
            StageScope sc(ST_GEMM_B0, st);
            if ((s = gemm_bf16(EPI_STORE, 0, dZ1, W1b, nheads * Mp, NFP, H, f16 ? 0 : (sp & 8) != 0, e, status, st,
                               m->gemm_bn, m->gemm_cps, f16)) != GM_OK)
                return fail(s, "tcgen05 GEMM B0 failed");
        }
        return GM_OK;
    }
    if (!from_l2) {
        e.bias = m->b1;
        e.out0 = w.A1;
        e.out1 = w.D1;
        StageScope sc(ST_GEMM_L1, st);
        gemm_f32(EPI_L1, m->d.activation, w.G, m->W1t, Mp, H, NFP, e, st);
    }
    e.bias = m->b2;
    e.out1 = nullptr;
    e.out0 = w.dZ2;
    e.head_stride = (size_t)Mp * H;
    {
        StageScope sc(ST_GEMM_L2, st);
        gemm_f32(l2, m->d.activation, w.A1, m->W2t, Mp, H, H, e, st);
    }
    e.out0 = w.dZ1;
    e.aux = w.D1;
    e.aux_rows = nheads > 1 ? Mp : 0;
    {
        StageScope sc(ST_GEMM_B1, st);
        gemm_f32(EPI_B1, 0, w.dZ2, m->W2, nheads * Mp, H, H, e, st);
    }
    e.out0 = w.dG;
    {
        StageScope sc(ST_GEMM_B0, st);
        gemm_f32(EPI_STORE, 0, w.dZ1, m->W1p, nheads * Mp, NFP, H, e, st);
    }
    return GM_OK;
}

// Energies, forces and virials of the model (the mean head for a shallow ensemble); with ens,
// the L2 epilogue also leaves every head's partial sums in w.nn_ens.
static gm_status energy_forces_pipeline(const gm_model *m, const gm_system *sys, const gm_nlist *nl, double *energy,
                                        float *forces, double *virial, EfWs &w, bool ens, int32_t *status,
                                        cudaStream_t st) {
    const int N = sys->n_atoms, B = sys->n_structures, H = m->H;
    const int Mp = round_up(N, TILE_M);
    gm_status s;
    // without the virial, the mixed path sums the energies inside its B1 GEMM or its cluster
    // network kernel (after the per-tile fused kernel the reduction kernel does)
    int cs = 1;
    const bool fused_energy = N > 0 && virial == nullptr && m->d.precision == GM_PREC_MIXED &&
                              mlp_form(m, ens, false, nullptr, N, &cs) != MLP_TILE;
    if (N > 0) {
        if ((s = forward_to_features(m, sys, nl, w, nullptr, nullptr, forces, status, st)) != GM_OK) return s;
        if ((s = network_fwd_bwd(m, sys, w, Mp, status, st, fused_energy ? energy : nullptr, nullptr, ens)) != GM_OK)
            return s;
        {
            // the fused network kernels (per tile or per cluster) leave dE/dG in their tiled layout
            StageScope sc(ST_CONTRACT_BWD, st);
            launch_contract_bwd(w.psi, w.dG, N, w.dpsi, st, mlp_form(m, ens, false, nullptr, N, &cs) != MLP_GEMMS);
        }
        PairArgs a = pair_args(m, sys, nl, w.pos_hi, w.pos_lo, status);
        StageScope sc(ST_FORCES, st);
        launch_forces(a, choose_forces_tpa(m, N), w.dpsi, forces, virial ? w.vir_atom : nullptr, st);
    }
    if (!fused_energy) {
        StageScope sc(ST_REDUCE, st);
        launch_struct_reduce(B, N, sys->atom_ptr, sys->species, m->S, m->sigma, m->mu, m->b3, w.nn_part, H / 32,
                             virial ? w.vir_atom : nullptr, w.red_acc, energy, virial, st);
    }
    return launch_status();
}

gm_status gm_energy_forces(const gm_model *m, const gm_system *sys, const gm_nlist *nl, double *energy, float *forces,
                           double *virial, void *ws, size_t ws_bytes, int32_t *status, struct CUstream_st *stream) {
    gm_status s = check_system(m, sys);
    if (s != GM_OK) return s;
    if ((s = check_nlist(sys, nl, true)) != GM_OK) return s;
    if (!energy || !status || (sys->n_atoms > 0 && !forces)) return fail(GM_ERR_ARG, "null output");
    Carve c(ws, ws_bytes);
    EfWs w = carve_ef(c, sys->n_structures, sys->n_atoms, m->H);
    if (!c.ok) return fail(GM_ERR_WORKSPACE, "workspace too small");
    return energy_forces_pipeline(m, sys, nl, energy, forces, virial, w, false, status, stream);
}

gm_status gm_energy_forces_ensemble(const gm_model *m, const gm_system *sys, const gm_nlist *nl, double *energy,
                                    float *forces, double *virial, double *energy_heads, double *energy_std,
                                    int32_t mode, float *forces_heads, float *force_std, void *ws, size_t ws_bytes,
                                    int32_t *status, struct CUstream_st *stream) {
    gm_status s = check_system(m, sys);
    if (s != GM_OK) return s;
    if ((s = check_nlist(sys, nl, true)) != GM_OK) return s;
    if (!energy || !status || (sys->n_atoms > 0 && !forces)) return fail(GM_ERR_ARG, "null output");
    if (mode != GM_ENS_MEAN_GRADIENT && mode != GM_ENS_JACOBIAN) return fail(GM_ERR_ARG, "bad ensemble force mode");
    if (mode == GM_ENS_MEAN_GRADIENT && (forces_heads || force_std))
        return fail(GM_ERR_ARG, "per-head forces and their spread need GM_ENS_JACOBIAN");
    if (!aligned(energy_heads, 8) || !aligned(energy_std, 8) || !aligned(forces_heads, 4) || !aligned(force_std, 4))
        return fail(GM_ERR_ARG, "misaligned ensemble output");
    const int N = sys->n_atoms, B = sys->n_structures, H = m->H, E = m->E;
    if (E < 2) return fail(GM_ERR_ARG, "the model has a single output head (n_ensemble <= 1)");
    Carve c(ws, ws_bytes);
    EfWs w = carve_ef(c, B, N, H, E);
    if (!c.ok) return fail(GM_ERR_WORKSPACE, "workspace too small");
    cudaStream_t st = stream;
    // (the head-energy accumulators are cleared with the structure sums by the position split)
    // the mean head: energies, forces (gradient of the mean energy) and virials, with every
    // head's partial sums written in the L2 epilogue
    if ((s = energy_forces_pipeline(m, sys, nl, energy, forces, virial, w, true, status, st)) != GM_OK) return s;
    {
        StageScope sc(ST_REDUCE, st);
        launch_ens_energy(B, N, E, sys->atom_ptr, sys->species, m->S, m->sigma, m->mu, m->b3e, w.nn_ens, H / 32,
                          (size_t)round_up(N, TILE_M), w.ens_acc, energy_heads, energy_std, st);
    }
    if (mode == GM_ENS_JACOBIAN && N > 0) {
        // every head's forces: the backward pass from L2 with that head's weights (the features,
        // the first layer and the moments of the mean pass are reused); the backward
        // contraction, the force pass and the two backward GEMMs of a chunk of heads run as one
        // launch each
        const int Mp = round_up(N, TILE_M);
        float *Fk = forces_heads ? forces_heads : w.Fk;
        PairArgs a = pair_args(m, sys, nl, w.pos_hi, w.pos_lo, status);
        const int hc = ens_head_chunk(E, N);
        for (int k0 = 0; k0 < E; k0 += hc) {
            const int kn = std::min(hc, E - k0);
            float *Fh = Fk + (size_t)k0 * N * 3;
            if (cudaMemsetAsync(Fh, 0, sizeof(float) * 3 * (size_t)N * kn, st) != cudaSuccess)
                return fail(GM_ERR_CUDA, "memset of the head forces failed");
            EfWs wh = w;                                // the chunk's stacked dZ2, dZ1 and dG rows
            wh.dZ2 = w.dZ2h;
            wh.dZ1 = w.dZ1h;
            wh.dG = w.dGh;
            if ((s = network_fwd_bwd(m, sys, wh, Mp, status, st, nullptr, m->w3e + (size_t)k0 * H, false, true,
                                     kn)) != GM_OK)
                return s;
            {
                StageScope sc(ST_CONTRACT_BWD, st);
                launch_contract_bwd(w.psi, w.dGh, N, w.dpsih, st, false, kn, (size_t)Mp * NFP);
            }
            StageScope sc(ST_FORCES, st);
            launch_forces(a, choose_forces_tpa(m, N * kn), w.dpsih, Fh, nullptr, st, kn);
        }
        if (force_std) launch_ens_force_std(N, E, Fk, force_std, st);
    }
    return launch_status();
}

// ------------------------------------------------------------------ molecular dynamics

static gm_status md_check(const gm_model *m, const gm_system *sys, const gm_nlist *nl, const gm_md_params *params,
                          const gm_md_state *st, const int32_t *status) {
    gm_status s = check_system(m, sys);
    if (s != GM_OK) return s;
    if ((s = check_nlist(sys, nl, false)) != GM_OK) return s;
    if (!status || !st) return fail(GM_ERR_ARG, "null status or state");
    if (md_check_params(params) != GM_OK) return fail(GM_ERR_ARG, "bad MD parameters");
    if (m->E > 1) return fail(GM_ERR_UNSUPPORTED, "MD of a shallow-ensemble model uses its mean; not implemented");
    if (!st->pos || !st->vel || !st->mass || !st->kinetic || !st->energy || !st->pos_ref || !st->chain ||
        (sys->n_atoms > 0 && !st->forces))
        return fail(GM_ERR_ARG, "null MD state field");
    if (st->pos != sys->pos) return fail(GM_ERR_ARG, "state->pos must be the system's positions");
    if (!aligned(st->vel, 8) || !aligned(st->mass, 8) || !aligned(st->forces, 4) || !aligned(st->energy, 8) ||
        !aligned(st->kinetic, 8) || !aligned(st->pos_ref, 8) || !aligned(st->chain, 8) || !aligned(st->n_builds, 8))
        return fail(GM_ERR_ARG, "misaligned MD state field");
    return GM_OK;
}

gm_status gm_md_init(const gm_model *m, const gm_system *sys, gm_nlist *nl, const gm_md_params *params,
                     gm_md_state *state, void *ws, size_t ws_bytes, int32_t *status, struct CUstream_st *stream) {
    gm_status s = md_check(m, sys, nl, params, state, status);
    if (s != GM_OK) return s;
    const int N = sys->n_atoms, B = sys->n_structures;
    Carve c(ws, ws_bytes);
    MdWs w = carve_md(c, B, N, m->H, nl->capacity);
    if (!c.ok) return fail(GM_ERR_WORKSPACE, "workspace too small");
    cudaStream_t st = stream;
    // chains at rest, accumulators at zero, and the skin flag set so that the kinetic pass
    // below records pos_ref and counts this build
    if (cudaMemsetAsync(state->chain, 0, sizeof(double) * 2 * GM_MD_MAX_CHAIN * B, st) != cudaSuccess ||
        cudaMemsetAsync(w.acc, 0, sizeof(unsigned long long) * reduce_acc_words(B), st) != cudaSuccess ||
        cudaMemsetAsync(w.flag, 0, sizeof(int32_t) * 64, st) != cudaSuccess ||
        cudaMemsetAsync(w.flag, 1, 1, st) != cudaSuccess)
        return fail(GM_ERR_CUDA, "memset of the MD state failed");
    {
        StageScope sc(ST_NEIGHBORS, st);
        if ((s = nl_build(*sys, m->d.r_cut + params->skin, m->S, *nl, w.nl, w.nl_bytes, status, st, m->nl)) != GM_OK)
            return fail(s, "neighbour build launch failed");
    }
    if ((s = energy_forces_pipeline(m, sys, nl, state->energy, state->forces, nullptr, w.ef, false, status, st)) != GM_OK)
        return s;
    gm_md_params nve = *params;
    nve.ensemble = GM_MD_NVE;     // kinetic energies only: no thermostat step here
    StageScope sc(ST_MD, st);
    md_kick_ke(N, B, sys->atom_ptr, sys->species, state->mass, state->forces, nve, 0, state->vel, state->pos,
               state->pos_ref, w.flag, w.acc, state->kinetic, state->chain, w.pending, state->n_builds, 1, status,
               st);
    return launch_status();
}

gm_status gm_md_run(const gm_model *m, const gm_system *sys, gm_nlist *nl, const gm_md_params *params,
                    gm_md_state *state, int32_t n_steps, void *ws, size_t ws_bytes, int32_t *status,
                    struct CUstream_st *stream) {
    gm_status s = md_check(m, sys, nl, params, state, status);
    if (s != GM_OK) return s;
    if (n_steps < 0) return fail(GM_ERR_ARG, "negative step count");
    const int N = sys->n_atoms, B = sys->n_structures;
    Carve c(ws, ws_bytes);
    MdWs w = carve_md(c, B, N, m->H, nl->capacity);
    if (!c.ok) return fail(GM_ERR_WORKSPACE, "workspace too small");
    cudaStream_t st = stream;
    if (cudaMemsetAsync(w.acc, 0, sizeof(unsigned long long) * reduce_acc_words(B), st) != cudaSuccess ||
        cudaMemsetAsync(w.flag, 0, sizeof(int32_t) * 64, st) != cudaSuccess)
        return fail(GM_ERR_CUDA, "memset of the MD words failed");
    const bool nvt = params->ensemble == GM_MD_NVT;
    const double r_list = m->d.r_cut + params->skin;
    for (int k = 0; k < n_steps; ++k) {
        {
            StageScope sc(ST_MD, st);
            if (nvt && k == 0) md_thermo(B, sys->atom_ptr, *params, state->chain, state->kinetic, w.pending, status, st);
            md_kick_drift(N, B, sys->atom_ptr, sys->species, state->mass, state->forces, nvt ? w.pending : nullptr,
                          *params, state->vel, state->pos, state->pos_ref, w.flag, status, st);
        }
        {
            StageScope sc(ST_NEIGHBORS, st);
            if ((s = nl_build(*sys, r_list, m->S, *nl, w.nl, w.nl_bytes, status, st, m->nl, w.flag)) != GM_OK)
                return fail(s, "neighbour build launch failed");
        }
        if ((s = energy_forces_pipeline(m, sys, nl, state->energy, state->forces, nullptr, w.ef, false, status, st)) !=
            GM_OK)
            return s;
        StageScope sc(ST_MD, st);
        md_kick_ke(N, B, sys->atom_ptr, sys->species, state->mass, state->forces, *params, 1, state->vel, state->pos,
                   state->pos_ref, w.flag, w.acc, state->kinetic, state->chain, w.pending, state->n_builds,
                   k == n_steps - 1, status, st);
    }
    if (nvt && n_steps > 0) {
        StageScope sc(ST_MD, st);
        md_finish(N, B, sys->atom_ptr, w.pending, state->vel, status, st);
    }
    return launch_status();
}

gm_status gm_descriptors(const gm_model *m, const gm_system *sys, const gm_nlist *nl, float *psi, float *features,
                         void *ws, size_t ws_bytes, int32_t *status, struct CUstream_st *stream) {
    gm_status s = check_system(m, sys);
    if (s != GM_OK) return s;
    if ((s = check_nlist(sys, nl, true)) != GM_OK) return s;
    if (!psi || !status) return fail(GM_ERR_ARG, "null output");
    if (!aligned(psi, 16)) return fail(GM_ERR_ARG, "psi must be 16-byte aligned");
    Carve c(ws, ws_bytes);
    EfWs w = carve_ef(c, sys->n_structures, sys->n_atoms, m->H);
    if (!c.ok) return fail(GM_ERR_WORKSPACE, "workspace too small");
    if (sys->n_atoms == 0) return GM_OK;
    return forward_to_features(m, sys, nl, w, psi, features, nullptr, status, stream);
}

gm_status gm_param_grad(const gm_model *m, const gm_system *sys, const gm_nlist *nl, const double *dL_dE,
                        const float *dL_dF, float *grad_theta, void *ws, size_t ws_bytes, int32_t *status,
                        struct CUstream_st *stream) {
    gm_status s = check_system(m, sys);
    if (s != GM_OK) return s;
    if ((s = check_nlist(sys, nl, true)) != GM_OK) return s;
    if (!dL_dE || !grad_theta || !status || (sys->n_atoms > 0 && !dL_dF)) return fail(GM_ERR_ARG, "null argument");
    if (m->E > 1)
        return fail(GM_ERR_UNSUPPORTED, "the parameter gradient of a shallow-ensemble model is not implemented");
    const int N = sys->n_atoms, B = sys->n_structures, H = m->H, S = m->S;
    Carve c(ws, ws_bytes);
    PgWs w = carve_pg(c, N, H, S);
    if (!c.ok) return fail(GM_ERR_WORKSPACE, "workspace too small");
    cudaStream_t st = stream;
    const ThetaOff o = theta_offsets(S, H);
    if (cudaMemsetAsync(grad_theta, 0, sizeof(float) * o.total, st) != cudaSuccess)
        return fail(GM_ERR_CUDA, "memset of the gradient failed");
    if (N == 0) return launch_status();
    const int Mp = round_up(N, TILE_M);
    const int act = m->d.activation;
    PairArgs a = pair_args(m, sys, nl, w.pos_hi, w.pos_lo, status);
    {   // primal and tangent moments, features and their tangents
        StageScope sc(ST_PG_PAIR_FWD, st);
        launch_split_pos(N, sys->pos, sys->species, w.pos_hi, w.pos_lo, nullptr, nullptr, 0, st);
        launch_moments(a, choose_tpa(m, N), w.psi, st);
        launch_moments_tangent(a, choose_tangent_tpa(m, N), dL_dF, w.psid, st);
        launch_contract_fwd_dual(w.psi, w.psid, N, Mp, w.GG, st);
    }
    {   // network forward (primal + tangent rows) and reverse
        StageScope sc(ST_PG_NETWORK, st);
        EpiArgs e{};
        // the four stacked-row GEMMs: FFMA in the FP32 path; tcgen05 on hi/lo BF16 copies of
        // the A operand in the mixed path (split passes as for the energy/force GEMMs)
        const bool mixed = m->d.precision == GM_PREC_MIXED;
        const int sp = m->pg_split_mask;
        // (the activation kernels write the hi/lo copy of the next GEMM's A operand themselves;
        // only the features need a conversion pass)
        auto mm = [&](int which, const float *A, const float *Bf, const __nv_bfloat16 *Bh, int N_, int K_,
                      float *out) -> gm_status {
            e.out0 = out;
            if (!mixed) {
                gemm_f32(EPI_STORE, 0, A, Bf, 2 * Mp, N_, K_, e, st);
                return GM_OK;
            }
            if (which == 0) split_bf16(A, 2 * Mp, K_, w.hl, st);
            return gemm_bf16(EPI_STORE, 0, w.hl, Bh, 2 * Mp, N_, K_, ((sp >> which) & 1) != 0, e, status, st,
                             m->gemm_bn, m->gemm_cps);
        };
        __nv_bfloat16 *hl = mixed ? w.hl : nullptr;
        gm_status gs;
        if ((gs = mm(0, w.GG, m->W1t, m->W1t_h, H, NFP, w.Z)) != GM_OK) return fail(gs, "network GEMM 1 failed");
        pg_act1(act, Mp, H, w.Z, m->b1, w.A1s, w.P1, w.Q1, w.Zd1, hl, st);
        if ((gs = mm(1, w.A1s, m->W2t, m->W2t_h, H, H, w.Z)) != GM_OK) return fail(gs, "network GEMM 2 failed");
        pg_act2(act, N, Mp, H, B, sys->atom_ptr, sys->species, S, dL_dE, m->sigma, m->w3, m->b2, m->b3, w.Z, w.Zb2s,
                w.Y3, w.t_sig, w.t_c, w.t_cs, hl, st);
        // a1 adjoints (primal, tangent)
        if ((gs = mm(2, w.Zb2s, m->W2, m->W2_h, H, H, w.Z)) != GM_OK) return fail(gs, "network GEMM 3 failed");
        pg_act1b(Mp, H, w.Z, w.P1, w.Q1, w.Zd1, w.Zb1s, hl, st);
        // feature adjoints
        if ((gs = mm(3, w.Zb1s, m->W1p, m->W1p_h, NFP, H, w.Gbs)) != GM_OK) return fail(gs, "network GEMM 4 failed");
        // weight and bias gradients
        wgrad(w.GG, NFP, w.Zb1s, H, 2 * Mp, NFP, H, NF, w.wg_part, grad_theta + o.W1, st);
        wgrad(w.A1s, H, w.Zb2s, H, 2 * Mp, H, H, H, w.wg_part, grad_theta + o.W2, st);
        const float *cs_in[3] = {w.Zb1s, w.Zb2s, w.Y3};
        float *const cs_out[3] = {grad_theta + o.b1, grad_theta + o.b2, grad_theta + o.w3};
        colsum3(Mp, H, cs_in, cs_out, w.wg_part, st);
        pg_tail(N, sys->species, S, w.t_sig, w.t_c, w.t_cs, w.wg_part, grad_theta + o.sigma, grad_theta + o.mu,
                grad_theta + o.b3, st);
    }
    {   // moment adjoints and the species-pair coefficient gradient
        StageScope sc(ST_PG_PAIR_BWD, st);
        launch_contract_bwd_dual(w.psi, w.psid, w.Gbs, N, Mp, w.psib, w.psidb, st);
        launch_pg_beta(a, dL_dF, w.psib, w.psidb, w.beta_part, st);
        pg_beta_reduce(pg_beta_blocks(N, S), S * S * NR * NB, (float)(1.0 / sqrt((double)NB)), w.beta_part,
                       grad_theta + o.beta, st);
    }
    return launch_status();
}

gm_status gm_force_matching_loss(const gm_system *sys, const double *energy, const double *energy_ref,
                                 const float *forces, const float *forces_ref, double w_energy, double w_forces,
                                 double *loss, double *dL_dE, float *dL_dF, int32_t *status,
                                 struct CUstream_st *stream) {
    if (!sys || !energy || !energy_ref || !loss || !dL_dE || !status || !sys->atom_ptr)
        return fail(GM_ERR_ARG, "null argument");
    if (sys->n_atoms > 0 && (!forces || !forces_ref || !dL_dF)) return fail(GM_ERR_ARG, "null force argument");
    launch_loss(sys->n_structures, sys->n_atoms, sys->atom_ptr, energy, energy_ref, forces, forces_ref, w_energy,
                w_forces, loss, dL_dE, dL_dF, stream);
    return launch_status();
}

void gm_profile_enable(int on) { g_prof = on != 0; }

void gm_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &p : g_pending) {
        g_event_pool.push_back(p.a);
        g_event_pool.push_back(p.b);
    }
    g_pending.clear();
    for (int q = 0; q < N_STAGES; ++q) {
        g_stage_ms[q] = 0.0;
        g_stage_cnt[q] = 0;
    }
    g_launches = 0;
}

void gm_profile_forget_graphs(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_graph_stages.clear();  // the events stay alive: a graph may still record them
}

int gm_profile_n_stages(void) { return N_STAGES; }

const char *gm_profile_stage_name(int s) {
    static const char *names[N_STAGES] = {"neighbors", "moments", "contract_fwd", "gemm_l1", "gemm_l2",
                                          "gemm_b1", "gemm_b0", "contract_bwd", "forces", "reduce",
                                          "pg_pair_fwd", "pg_network", "pg_pair_bwd", "nl_bin", "nl_count",
                                          "nl_scan", "nl_fill", "nl_coop", "md_integrate", "mlp_fused"};
    return (s >= 0 && s < N_STAGES) ? names[s] : "";
}

gm_status gm_profile_collect(double *stage_ms, int64_t *stage_count, int n_stages, int64_t *kernel_launches) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &p : g_pending) {
        float ms = 0.0f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            g_stage_ms[p.stage] += ms;
            g_stage_cnt[p.stage] += 1;
        }
        g_event_pool.push_back(p.a);
        g_event_pool.push_back(p.b);
    }
    g_pending.clear();
    for (auto &p : g_graph_stages) {
        float ms = 0.0f;
        if (cudaEventQuery(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            g_stage_ms[p.stage] += ms;
            g_stage_cnt[p.stage] += 1;
        }
    }
    for (int q = 0; q < n_stages && q < N_STAGES; ++q) {
        if (stage_ms) stage_ms[q] = g_stage_ms[q];
        if (stage_count) stage_count[q] = g_stage_cnt[q];
    }
    if (kernel_launches) *kernel_launches = g_launches;
    return GM_OK;
}

gm_status gm_status_clear(int32_t *status, struct CUstream_st *stream) {
    if (!status) return fail(GM_ERR_ARG, "null status");
    if (cudaMemsetAsync(status, 0, sizeof(int32_t), stream) != cudaSuccess) return fail(GM_ERR_CUDA, "memset failed");
    return GM_OK;
}

const char *gm_status_string(gm_status s) {
    switch (s) {
    case GM_OK: return "ok";
    case GM_ERR_ARG: return "invalid argument";
    case GM_ERR_CAPACITY: return "neighbour list capacity exceeded";
    case GM_ERR_UNSUPPORTED: return "unsupported configuration";
    case GM_ERR_CUDA: return "CUDA error";
    case GM_ERR_TIMEOUT: return "device wait timed out";
    case GM_ERR_SPECIES: return "species index out of range";
    case GM_ERR_WORKSPACE: return "workspace too small";
    }
    return "unknown status";
}

const char *gm_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
