// gm_gemm_tc.cu -- host side of the tcgen05 network kernels: TMA tensor maps (cached by base,
// shape and box), tile choice and launch of the GEMM (gm_gemm_tc.cuh), of the four layers
// fused per tile (gm_mlp_fused.cuh) and per thread-block cluster (gm_mlp_cluster.cuh).
#include <cudaTypedefs.h>

#include <map>
#include <mutex>
#include <tuple>

#include "gm_gemm_tc.cuh"
#include "gm_mlp_cluster.cuh"

namespace gm {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

using MapKey = std::tuple<const void *, int, int, int>;
std::mutex g_map_mu;
std::map<MapKey, CUtensorMap> g_maps;

// 2-D BF16 tensor [rows][inner] (inner contiguous), box 64 x box_rows, 128-byte swizzle.
bool tensor_map(const void *base, int inner, int rows, int box_rows, CUtensorMap *out) {
    const MapKey key{base, inner, rows, box_rows};
    std::lock_guard<std::mutex> lk(g_map_mu);
    auto it = g_maps.find(key);
    if (it != g_maps.end()) {
        *out = it->second;
        return true;
    }
    auto fn = encode_fn();
    if (!fn) return false;
    CUtensorMap m;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)inner * 2};
    cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    if (g_maps.size() > 256) g_maps.clear();
    g_maps.emplace(key, m);
    *out = m;
    return true;
}

template <int BN, int EPI, int ACT, int CPS>
cudaError_t launch_tc(const CUtensorMap &ma, const CUtensorMap &mb, int M, int N, int K, int split,
                      const EpiArgs &e, int32_t *status, cudaStream_t st, int f16) {
    static PerDeviceOnce attr_set;
    const size_t smem = tc::smem_bytes_for(BN, CPS);
    if (attr_set.first()) {
        cudaError_t err = cudaFuncSetAttribute(tc::k_gemm_tc<BN, EPI, ACT, CPS>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
    }
    dim3 grid(N / BN, M / tc::BM);
    launch_pdl(tc::k_gemm_tc<BN, EPI, ACT, CPS>, grid, dim3(256), smem, st, ma, mb, M, N, K, split, e, status, f16);
    return cudaPeekAtLastError();
}

template <int BN, int CPS>
cudaError_t dispatch_epi(int epi, int act, const CUtensorMap &ma, const CUtensorMap &mb, int M, int N, int K,
                         int split, const EpiArgs &e, int32_t *status, cudaStream_t st, int f16) {
    switch (epi) {
    case EPI_L1:
        return act == 0 ? launch_tc<BN, EPI_L1, 0, CPS>(ma, mb, M, N, K, split, e, status, st, f16)
                        : launch_tc<BN, EPI_L1, 1, CPS>(ma, mb, M, N, K, split, e, status, st, f16);
    case EPI_L2:
        return act == 0 ? launch_tc<BN, EPI_L2, 0, CPS>(ma, mb, M, N, K, split, e, status, st, f16)
                        : launch_tc<BN, EPI_L2, 1, CPS>(ma, mb, M, N, K, split, e, status, st, f16);
    case EPI_L2E:
        return act == 0 ? launch_tc<BN, EPI_L2E, 0, CPS>(ma, mb, M, N, K, split, e, status, st, f16)
                        : launch_tc<BN, EPI_L2E, 1, CPS>(ma, mb, M, N, K, split, e, status, st, f16);
    case EPI_L2H:
        return act == 0 ? launch_tc<BN, EPI_L2H, 0, CPS>(ma, mb, M, N, K, split, e, status, st, f16)
                        : launch_tc<BN, EPI_L2H, 1, CPS>(ma, mb, M, N, K, split, e, status, st, f16);
    case EPI_B1: return launch_tc<BN, EPI_B1, 0, CPS>(ma, mb, M, N, K, split, e, status, st, f16);
    default: return launch_tc<BN, EPI_STORE, 0, CPS>(ma, mb, M, N, K, split, e, status, st, f16);
    }
}

template <int BN>
cudaError_t dispatch_cps(int cps, int epi, int act, const CUtensorMap &ma, const CUtensorMap &mb, int M, int N,
                         int K, int split, const EpiArgs &e, int32_t *status, cudaStream_t st, int f16) {
    return cps == 2 ? dispatch_epi<BN, 2>(epi, act, ma, mb, M, N, K, split, e, status, st, f16)
                    : dispatch_epi<BN, 1>(epi, act, ma, mb, M, N, K, split, e, status, st, f16);
}

}  // namespace

int tc_choose_bn(int M, int N, int forced) {
    if (forced == 64 || forced == 128 || forced == 256) return (N % forced == 0) ? forced : 64;
    const long long tiles_m = M / tc::BM;
    if (N % 256 == 0 && tiles_m * (N / 256) >= 148) return 256;
    if (N % 128 == 0 && tiles_m * (N / 128) >= 148) return 128;
    if (N % 128 == 0 && tiles_m * (N / 64) > 2 * 148) return 128;
    return 64;
}

// CTAs per SM: two (halved stage ring) once there are enough tiles to fill the GPU twice
int tc_choose_cps(int M, int N, int bn, int forced) {
    if (forced == 1 || forced == 2) return forced;
    const long long tiles = (long long)(M / tc::BM) * (N / bn);
    return tiles >= 2 * 148 ? 2 : 1;
}

gm_status gemm_bf16(int epi, int act, const __nv_bfloat16 *A, const __nv_bfloat16 *B, int M, int N, int K, int split,
                    const EpiArgs &e, int32_t *status, cudaStream_t st, int forced_bn, int forced_cps, int f16) {
    if (M <= 0) return GM_OK;
    if (M % tc::BM || K % tc::BK || N % 64 || M / tc::BM > 65535) return GM_ERR_UNSUPPORTED;
    if (f16 && split) return GM_ERR_UNSUPPORTED;      // FP16 operands are read in one pass
    const int bn = tc_choose_bn(M, N, forced_bn);
    const int cps = tc_choose_cps(M, N, bn, forced_cps);
    CUtensorMap ma, mb;
    // operands are [rows][2K] hi/lo pairs
    if (!tensor_map(A, 2 * K, M, tc::BM, &ma) || !tensor_map(B, 2 * K, N, bn, &mb)) return GM_ERR_CUDA;
    cudaError_t err;
    switch (bn) {
    case 256: err = dispatch_cps<256>(cps, epi, act, ma, mb, M, N, K, split, e, status, st, f16); break;
    case 128: err = dispatch_cps<128>(cps, epi, act, ma, mb, M, N, K, split, e, status, st, f16); break;
    default: err = dispatch_cps<64>(cps, epi, act, ma, mb, M, N, K, split, e, status, st, f16); break;
    }
    note_launches(1);
    return err == cudaSuccess ? GM_OK : GM_ERR_CUDA;
}

namespace {
template <int H, int ACT>
cudaError_t launch_fused(const CUtensorMap *maps, const tc::FusedArgs &f, int ctas, int32_t *status, cudaStream_t st) {
    using Sh = tc::FusedShape<H>;
    static PerDeviceOnce attr_set;
    if (attr_set.first()) {
        cudaError_t err = cudaFuncSetAttribute(tc::k_mlp_fused<H, ACT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)Sh::SMEM);
        if (err != cudaSuccess) return err;
    }
    // persistent: one CTA per SM (or the requested number), tiles dealt round-robin
    const int tiles = f.M / tc::BM, want = ctas > 0 ? ctas : device_sm_count();
    launch_pdl(tc::k_mlp_fused<H, ACT>, dim3(tiles < want ? tiles : want), dim3(320), Sh::SMEM, st, maps[0],
               maps[1], maps[2], maps[3], maps[4], f, status);
    return cudaPeekAtLastError();
}
}  // namespace

namespace {
// launch configuration of the cluster kernel: CS CTAs per 128-row tile
template <int H, int CS, int ACT>
cudaLaunchConfig_t cluster_cfg(int M, cudaStream_t st, cudaLaunchAttribute *attr) {
    using Sh = tc::ClusterShape<H, CS>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(M / tc::BM * CS));
    cfg.blockDim = dim3(320);
    cfg.dynamicSmemBytes = Sh::SMEM;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cfg;
}

// clusters of the kernel the device keeps resident at once (0: it cannot launch); per device
template <int H, int CS, int ACT>
int cluster_capacity() {
    static int cap[64];
    static bool known[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (known[dev]) return cap[dev];
    using Sh = tc::ClusterShape<H, CS>;
    int n = 0;
    if (cudaFuncSetAttribute(tc::k_mlp_cluster<H, CS, ACT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Sh::SMEM) == cudaSuccess) {
        cudaLaunchAttribute attr[2];
        cudaLaunchConfig_t cfg = cluster_cfg<H, CS, ACT>(tc::BM, nullptr, attr);
        cfg.numAttrs = 1;   // the occupancy query takes the cluster shape alone
        if (cudaOccupancyMaxActiveClusters(&n, tc::k_mlp_cluster<H, CS, ACT>, &cfg) != cudaSuccess) n = 0;
    }
    cudaGetLastError();
    cap[dev] = n;
    known[dev] = true;
    return n;
}

template <int H, int CS, int ACT>
cudaError_t launch_cluster(const CUtensorMap *maps, const tc::ClusterArgs &f, int32_t *status, cudaStream_t st) {
    if (cluster_capacity<H, CS, ACT>() <= 0) return cudaErrorNotSupported;   // also sets the smem attribute
    cudaLaunchAttribute attr[2];
    cudaLaunchConfig_t cfg = cluster_cfg<H, CS, ACT>(f.M, st, attr);
    return cudaLaunchKernelEx(&cfg, tc::k_mlp_cluster<H, CS, ACT>, maps[0], maps[1], maps[2], maps[3], maps[4],
                              maps[5], maps[6], maps[7], f, status);
}

template <int H, int CS>
cudaError_t launch_cluster_act(int act, const CUtensorMap *maps, const tc::ClusterArgs &f, int32_t *status,
                               cudaStream_t st) {
    return act == 0 ? launch_cluster<H, CS, 0>(maps, f, status, st) : launch_cluster<H, CS, 1>(maps, f, status, st);
}
}  // namespace

bool mlp_fused_supported(int H) { return H == 128 || H == 256 || H == 512; }

bool mlp_cluster_supported(int H, int cs) {
    return mlp_fused_supported(H) && (cs == 2 || cs == 4 || cs == 8) && H / cs >= 64;
}

int mlp_cluster_capacity(int act, int H, int cs) {
    if (!mlp_cluster_supported(H, cs)) return 0;
    const bool silu = act != 0;
#define GM_CAP(h, c) if (H == h && cs == c) return silu ? cluster_capacity<h, c, 1>() : cluster_capacity<h, c, 0>();
    GM_CAP(512, 8) GM_CAP(512, 4) GM_CAP(512, 2) GM_CAP(256, 4) GM_CAP(256, 2) GM_CAP(128, 2)
#undef GM_CAP
    return 0;
}

gm_status mlp_cluster(int act, int M, int H, int cs, const __nv_bfloat16 *G, const __nv_bfloat16 *W1t,
                      const __nv_bfloat16 *W2t, const __half *W2, const __half *W1p, const FusedMlpArgs &a,
                      int32_t *status, cudaStream_t st) {
    if (M <= 0) return GM_OK;
    if (M % tc::BM || !mlp_cluster_supported(H, cs) || (long long)(M / tc::BM) * cs > 65535)
        return GM_ERR_UNSUPPORTED;
    const int w = H / cs, wg = NFP / cs;
    if (!a.xa1 || !a.xdz2 || !a.xdz1) return GM_ERR_ARG;
    CUtensorMap maps[8];
    // operands in the [rows][2K] layout of the split path (hi slots read); the three gather
    // arrays in the same layout
    if (!tensor_map(G, 2 * NFP, M, tc::BM, &maps[0]) || !tensor_map(W1t, 2 * NFP, H, w, &maps[1]) ||
        !tensor_map(W2t, 2 * H, H, w, &maps[2]) || !tensor_map(W2, 2 * H, H, w, &maps[3]) ||
        !tensor_map(W1p, 2 * H, NFP, wg, &maps[4]) || !tensor_map(a.xa1, 2 * H, M, tc::BM, &maps[5]) ||
        !tensor_map(a.xdz2, 2 * H, M, tc::BM, &maps[6]) || !tensor_map(a.xdz1, 2 * H, M, tc::BM, &maps[7]))
        return GM_ERR_CUDA;
    tc::ClusterArgs f;
    f.M = M;
    f.n_atoms = a.n_atoms;
    f.n_species = a.n_species;
    f.species = a.species;
    f.b1 = a.b1;
    f.b2 = a.b2;
    f.w3 = a.w3;
    f.sigma = a.sigma;
    f.D1 = a.D1;
    f.nn_part = a.nn_part;
    f.dG = a.dG;
    f.debug_stall = a.debug_stall;
    f.atom_ptr = a.atom_ptr;
    f.n_structures = a.n_structures;
    f.mu = a.mu;
    f.b3 = a.b3;
    f.red_acc = a.red_acc;
    f.energy = a.energy;
    cudaError_t err = cudaErrorNotSupported;
#define GM_LAUNCH(h, c) if (H == h && cs == c) err = launch_cluster_act<h, c>(act, maps, f, status, st);
    GM_LAUNCH(512, 8) GM_LAUNCH(512, 4) GM_LAUNCH(512, 2) GM_LAUNCH(256, 4) GM_LAUNCH(256, 2) GM_LAUNCH(128, 2)
#undef GM_LAUNCH
    note_launches(1);
    if (err == cudaErrorNotSupported) return GM_ERR_UNSUPPORTED;
    return err == cudaSuccess ? GM_OK : GM_ERR_CUDA;
}

gm_status mlp_fused(int act, int M, int H, const __nv_bfloat16 *G, const __nv_bfloat16 *W1t, const __nv_bfloat16 *W2t,
                    const __half *W2, const __half *W1p, const FusedMlpArgs &a, int32_t *status, cudaStream_t st) {
    if (M <= 0) return GM_OK;
    if (M % tc::BM || !mlp_fused_supported(H) || M / tc::BM > 65535) return GM_ERR_UNSUPPORTED;
    const int chunk = H >= 256 ? 256 : H;
    CUtensorMap maps[5];
    // operands in the [rows][2K] layout of the split path (hi slots read)
    if (!tensor_map(G, 2 * NFP, M, tc::BM, &maps[0]) || !tensor_map(W1t, 2 * NFP, H, chunk, &maps[1]) ||
        !tensor_map(W2t, 2 * H, H, chunk, &maps[2]) || !tensor_map(W2, 2 * H, H, chunk, &maps[3]) ||
        !tensor_map(W1p, 2 * H, NFP, 128, &maps[4]))
        return GM_ERR_CUDA;
    tc::FusedArgs f;
    f.M = M;
    f.n_atoms = a.n_atoms;
    f.n_species = a.n_species;
    f.species = a.species;
    f.b1 = a.b1;
    f.b2 = a.b2;
    f.w3 = a.w3;
    f.sigma = a.sigma;
    f.D1 = a.D1;
    f.nn_part = a.nn_part;
    f.dG = a.dG;
    f.debug_stall = a.debug_stall;
    cudaError_t err;
    switch (H) {
    case 128: err = act == 0 ? launch_fused<128, 0>(maps, f, a.ctas, status, st) : launch_fused<128, 1>(maps, f, a.ctas, status, st); break;
    case 256: err = act == 0 ? launch_fused<256, 0>(maps, f, a.ctas, status, st) : launch_fused<256, 1>(maps, f, a.ctas, status, st); break;
    default: err = act == 0 ? launch_fused<512, 0>(maps, f, a.ctas, status, st) : launch_fused<512, 1>(maps, f, a.ctas, status, st); break;
    }
    note_launches(1);
    return err == cudaSuccess ? GM_OK : GM_ERR_CUDA;
}

}  // namespace gm
