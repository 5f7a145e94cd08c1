/*
 * gm.h -- C ABI of libgm: Gaussian Moment Neural Network (GMNN) energies, forces and
 * force-matching parameter gradients on an NVIDIA B300 (sm_103a).
 *
 * The model (paper: "Apax", section "Machine Learning Interatomic Potentials"):
 *   E(S)         = sum_i E_i                                     Eq. energy_sum
 *   Psi_{i,L,s}  = sum_{j != i} R_{Zi,Zj,s}(r_ij) rhat_ij^{(x)L}  Eq. basis_fn, L = 0..3
 *   G_i          = full tensor contractions of Psi_i             Eq. contraction
 *   E_i          = sigma_{Zi} NN(G_i) + mu_{Zi}                  Eq. scale_shift
 *   F_i          = -dE/dr_i, virial = -dE/d(strain)              (forces and virials as
 *                                                                 gradients, section
 *                                                                 "Model Abstractions")
 * Readings where the paper is silent:
 *   radial basis  Phi_k(r) = exp(-gamma (r - mu_k)^2), mu_k = r_min + k (r_cut - r_min)/(n_basis-1),
 *                 gamma = n_basis^2 / r_cut^2 ("equidistant Gaussians")
 *   cutoff        f_c(r) = (cos(pi r / r_cut) + 1)/2 for r < r_cut
 *   radial fns    R_s(r) = f_c(r) n_basis^{-1/2} sum_k beta[Zi][Zj][s][k] Phi_k(r), ordered pair
 *   features      360 invariants in 8 families (Psi0; Psi1.Psi1; Psi2:Psi2; Psi3:Psi3;
 *                 tr Psi2 Psi2 Psi2; Psi1 Psi2 Psi1; Psi3 Psi3 Psi2; Psi1 Psi3 Psi2), each
 *                 with its radial-index symmetry removed, family-major, lexicographic in
 *                 (s1, s2, s3)
 *   network       NN = w3 . phi(W2^T phi(W1^T G + b1) + b2) + b3, phi = tanh or SiLU
 *   neighbours    all (i, j, n) with |r'_j - r'_i + n.cell| < r_cut, except (j == i, n == 0);
 *                 periodic self-images count; r' are positions wrapped into the cell
 *
 * Conventions (every entry point):
 *   - Units: Angstrom and eV.  Energies and virials FP64; forces FP32 (eV/A).
 *   - The caller owns every buffer.  Entry points never allocate or free memory, except
 *     gm_model_create / gm_model_destroy, which own the model's repacked weight copies.
 *   - Device pointers are CUDA global memory of the current device.  All work is
 *     enqueued on `stream` (a cudaStream_t, passed as struct CUstream_st*), which must
 *     belong to the current device; calls do not synchronise the host.
 *   - The synchronous return value reports argument, shape and launch errors only.
 *     Conditions found on the device are written to *status_dev (an int32 the caller
 *     zeroes before a step): the first error wins; later kernels of the same step see a
 *     non-zero status and skip their work.  The caller reads it after synchronising.
 *   - Version 1 supports orthorhombic, fully periodic cells, n_basis = 7, n_radial = 5
 *     and 64 <= n_hidden <= 512 with n_hidden % 64 == 0; anything else returns
 *     GM_ERR_UNSUPPORTED (host-detectable) or writes it to *status_dev (cell shape).
 */
#ifndef GM_H
#define GM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st; /* cudaStream_t is struct CUstream_st* */

#if defined(__GNUC__)
#define GM_API __attribute__((visibility("default")))
#else
#define GM_API
#endif

typedef enum {
    GM_OK = 0,
    GM_ERR_ARG = 1,         /* NULL pointer, bad size or misaligned pointer */
    GM_ERR_CAPACITY = 2,    /* neighbour list needs more than nl->capacity pairs */
    GM_ERR_UNSUPPORTED = 3, /* configuration outside version 1 (see above) */
    GM_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed */
    GM_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    GM_ERR_SPECIES = 6,     /* a species index outside [0, n_species) */
    GM_ERR_WORKSPACE = 7    /* ws_bytes smaller than gm_workspace_size() */
} gm_status;

typedef enum { GM_ACT_TANH = 0, GM_ACT_SILU = 1 } gm_activation;

/* Radial basis (section "Machine Learning Interatomic Potentials" names both):
 *   GM_BASIS_GAUSSIAN  equidistant Gaussians (the reading above)
 *   GM_BASIS_BESSEL    Bessel-like functions of Kocer et al.,
 *                      f_k(r) = a_k [j0((k+1) pi r/r_cut) + j0((k+2) pi r/r_cut)], j0(x) = sin(x)/x,
 *                      a_k = (-1)^k sqrt(2) pi r_cut^(-3/2) (k+1)(k+2) / sqrt((k+1)^2 + (k+2)^2),
 *                      with the same cutoff f_c and n_basis^(-1/2) normalisation; r_min unused */
typedef enum { GM_BASIS_GAUSSIAN = 0, GM_BASIS_BESSEL = 1 } gm_basis;

/* Most shallow-ensemble output heads a model may have. */
#define GM_MAX_ENSEMBLE 32

typedef enum {
    GM_PREC_FP32 = 0,  /* moments, contractions and network in FP32 (FFMA) */
    GM_PREC_MIXED = 1  /* network GEMMs in BF16 on tcgen05 tensor cores with FP32
                          accumulation; everything else as GM_PREC_FP32 */
} gm_precision;

/* Largest system (all structures of a batch together) one call takes: the network GEMMs of
 * the parameter gradient stack two rows per atom in tiles of 128 rows, and a launch grid
 * has at most 65535 rows of tiles. */
#define GM_MAX_ATOMS 4000000

typedef struct {
    int32_t n_species;  /* S, 1..16 */
    int32_t n_basis;    /* radial basis functions (7) */
    int32_t n_radial;   /* radial functions (5, giving 360 features) */
    int32_t n_hidden;   /* H, width of both hidden layers */
    int32_t activation; /* gm_activation */
    int32_t precision;  /* gm_precision */
    double r_min;       /* first Gaussian centre (A) */
    double r_cut;       /* cutoff radius (A) */
    int32_t basis;      /* gm_basis; 0 (zero-initialised) = GM_BASIS_GAUSSIAN */
    int32_t n_ensemble; /* shallow-ensemble output heads N_ens (section "Uncertainty
                           Quantification"): 0 or 1 = one head, up to GM_MAX_ENSEMBLE */
} gm_model_desc;

typedef struct gm_model gm_model; /* opaque */

/* A batch of B periodic structures, N atoms in total (ragged, no padding). */
typedef struct {
    int32_t n_structures;     /* B >= 1 */
    int32_t n_atoms;          /* 0 <= N <= GM_MAX_ATOMS, else GM_ERR_UNSUPPORTED */
    const int32_t *atom_ptr;  /* device [B+1]; structure b owns atoms atom_ptr[b]..atom_ptr[b+1]-1 */
    const double *pos;        /* device [N][3] Cartesian positions (any image) */
    const int32_t *species;   /* device [N], 0 <= species < n_species */
    const double *cell;       /* device [B][3][3], rows are lattice vectors */
    const uint8_t *pbc;       /* device [B][3] periodic flags (version 1: all 1) */
} gm_system;

/* CSR neighbour list over the batch's global atom indices.  Within row i the pairs are
 * ordered by stencil cell, then by neighbour index (deterministic). */
typedef struct {
    int64_t capacity;   /* entries available in col and shift */
    int32_t *row_ptr;   /* device [N+1] */
    int32_t *col;       /* device [capacity]: neighbour atom j */
    int8_t *shift;      /* device [capacity][4]: (n0, n1, n2, 0); the displacement is
                           r_j - r_i + n0 a + n1 b + n2 c with the caller's positions */
    int64_t *n_pairs;   /* device scalar: number of pairs found (also set on overflow) */
} gm_nlist;

/* Workspace kinds for gm_workspace_size.  For GM_OP_NEIGHBORS and nl_capacity > 0 the size
 * includes a search slab of 4 x (1.25 x capacity / n_atoms + 16, rounded up to 32) bytes per
 * atom, which lets the build test every candidate pair once; with nl_capacity = 0 it is the
 * minimum, without the slab.  gm_build_neighbors accepts any workspace of at least the
 * minimum and uses the slab when it fits (else it tests the candidates twice: count, then
 * fill). */
enum { GM_OP_NEIGHBORS = 0, GM_OP_ENERGY_FORCES = 1, GM_OP_PARAM_GRAD = 2, GM_OP_MD = 3 };

/* Number of FP32 parameters.  Flat layout of theta, in this order:
 *   beta[S][S][n_radial][n_basis], W1[360][H], b1[H], W2[H][H], b2[H], w3[H][E], b3[E],
 *   sigma[S], mu[S]   (row-major; W1 maps features to the first hidden layer; E = the
 *   number of output heads, 1 unless desc.n_ensemble > 1). */
GM_API int64_t gm_param_count(const gm_model_desc *desc);

/* Create a model handle (allocates its device weight copies on the current device).
 * Errors: GM_ERR_ARG, GM_ERR_UNSUPPORTED, GM_ERR_CUDA. */
GM_API gm_status gm_model_create(const gm_model_desc *desc, gm_model **out);

/* Copy theta (device, FP32, gm_param_count entries, layout above) into the model and
 * repack the network weights for the kernels (transposed and padded, FP32 and BF16).
 * Asynchronous on `stream`; theta may be reused once the stream reaches this point. */
GM_API gm_status gm_model_set_params(gm_model *m, const float *theta_dev, struct CUstream_st *stream);

GM_API void gm_model_destroy(gm_model *m);

/* Tuning knobs of a model (they change speed, not results beyond rounding; the neighbour
 * knobs change nothing in the list):
 *   GM_TUNE_PAIR_TPA    lanes per atom in the pair kernels: 0 = by system size, or 1, 2, 4, 8, 16, 32
 *                       (the force kernel too, unless GM_TUNE_FORCES_TPA is set; with 2 and 4 the
 *                       moments kernel splits an atom's components over lane pairs)
 *   GM_TUNE_FORCES_TPA  lanes per atom of the force kernel alone: 0 = as GM_TUNE_PAIR_TPA (or by
 *                       size when that is 0), or 1, 2, 4, 8, 16, 32
 *   GM_TUNE_SPLIT_MASK  mixed path: network GEMMs that run with hi/lo split-BF16 operands
 *                       (three tensor-core passes) -- bit 1 first layer, 2 second layer,
 *                       4 and 8 the two backward GEMMs; default 12 (backward GEMMs), which
 *                       keeps forces within 2e-3 of the FP64 result
 *   GM_TUNE_F16_BACKWARD  mixed path: 1 (default) runs the two backward GEMMs of
 *                       gm_energy_forces on FP16 operands in one tensor-core pass (their
 *                       operands, dE/dz and the weights, are bounded, and FP16's 11-bit
 *                       significand keeps forces within 2e-3), 0 on BF16 with the split mask
 *   GM_TUNE_FUSED_MLP   mixed path: 1 runs the four network GEMMs of gm_energy_forces as one
 *                       tcgen05 kernel over 128-atom tiles, the layer activations kept on chip
 *                       (widths 128, 256 and 512, with the FP16 backward and no split in the
 *                       forward layers); 0: four GEMM launches; 2 (default): by size -- four
 *                       launches below 16 tiles, then a cluster per tile (GM_TUNE_MLP_CLUSTER,
 *                       2 or 4 CTAs) while all its CTAs fit on the GPU at once, else one CTA
 *                       per tile
 *   GM_TUNE_MLP_CLUSTER mixed path, fused network: CTAs sharing one 128-atom tile along the
 *                       hidden width (a thread-block cluster that all-gathers each layer's
 *                       activations in shared memory): 0 = by size (default), 1 = the per-tile
 *                       kernel (one CTA runs whole tiles), 2, 4 or 8 (hidden width / CTAs at least
 *                       64); a size the device
 *                       cannot launch falls back to the four GEMM launches
 *   GM_TUNE_MLP_CTAS    mixed path, one-CTA-per-tile fused network: CTAs of its persistent
 *                       launch, each taking every CTAs-th tile; 0 = one per SM (default), else
 *                       1..4096 (at most the number of tiles)
 *   GM_TUNE_PG_SPLIT_MASK  mixed path: the same bits for the four network GEMMs of
 *                       gm_param_grad (forward, forward, backward, backward on the stacked
 *                       primal and tangent rows); default 15 (all split), which keeps every
 *                       parameter group's gradient within 1e-5 relative L2 of the FP64 result
 *                       (12 gave 7e-3 on the scale parameters)
 *   GM_TUNE_GEMM_BN     mixed path: tensor-core tile width 64, 128 or 256 (0 = by size)
 *   GM_TUNE_GEMM_CPS    mixed path: tensor-core GEMM blocks resident per SM, 1 or 2 (two halve
 *                       the operand ring and overlap one block's epilogue with the other's
 *                       main loop; 0 = two when the tiles fill the GPU twice)
 *   GM_TUNE_NL_MODE     neighbour build as one cooperative launch (GM_NL_MODE_AUTO, the
 *                       default when the device supports it) or one launch per phase
 *                       (GM_NL_MODE_PHASES)
 *   GM_TUNE_NL_SPLIT    work items sharing one home cell in the neighbour search: 0 = by size, 1..16
 *   GM_TUNE_NL_BLOCKS   blocks of the cooperative neighbour launch: 0 = by size, else 1..4096
 *                       (capped at what the device keeps resident)
 *   GM_TUNE_NL_TWO_PASS 1: count-then-fill neighbour search even when the workspace holds the
 *                       search slab (0, the default: one search pass and a compaction)
 *   GM_TUNE_NL_ITEMS    neighbour search work items: 0 = by size (small systems whose boxes are
 *                       all at least 2 r_cut long: brute force over each structure's atoms,
 *                       same rows), 1 = one home cell (part) per block with shared staging,
 *                       2 = one per warp, 3 = brute force where possible, else as 0
 *   GM_TUNE_DEBUG_STALL 0 (default).  For tests of failure reporting only: 1 makes block 0 of
 *                       the cooperative neighbour build return before the first grid barrier,
 *                       so the other blocks' bounded waits run out; 2 makes the first network
 *                       GEMM of gm_energy_forces (mixed path), or the fused network kernel where
 *                       that runs, issue no operand loads, so its MMA and epilogue waits run
 *                       out.  Either way GM_ERR_TIMEOUT is written to
 *                       *status_dev after about a second and every block returns; nothing
 *                       asynchronous is in flight when a wait gives up, and the next call with
 *                       the knob at 0 is unaffected.
 * Errors: GM_ERR_ARG for an unknown key or value. */
enum { GM_TUNE_PAIR_TPA = 0, GM_TUNE_SPLIT_MASK = 1, GM_TUNE_GEMM_BN = 2, GM_TUNE_NL_MODE = 3, GM_TUNE_NL_SPLIT = 4,
       GM_TUNE_NL_BLOCKS = 5, GM_TUNE_NL_TWO_PASS = 6, GM_TUNE_NL_ITEMS = 7, GM_TUNE_GEMM_CPS = 8,
       GM_TUNE_PG_SPLIT_MASK = 9, GM_TUNE_DEBUG_STALL = 10, GM_TUNE_F16_BACKWARD = 11,
       GM_TUNE_FUSED_MLP = 12, GM_TUNE_FORCES_TPA = 13, GM_TUNE_MLP_CLUSTER = 14,
       GM_TUNE_MLP_CTAS = 15 };
enum { GM_NL_MODE_AUTO = 0, GM_NL_MODE_PHASES = 1 };
GM_API gm_status gm_model_set_tuning(gm_model *m, int32_t key, int32_t value);

/* Lanes per atom the moments kernels use for a system of n_atoms atoms: the GM_TUNE_PAIR_TPA
 * setting, or (when it is 0) the library's choice by size.  -1 for a null model or a
 * negative n_atoms. */
GM_API int32_t gm_model_pair_lanes(const gm_model *m, int32_t n_atoms);
/* The same for the force kernel (GM_TUNE_FORCES_TPA, else GM_TUNE_PAIR_TPA, else by size). */
GM_API int32_t gm_model_force_lanes(const gm_model *m, int32_t n_atoms);

/* Bytes of device memory the model handle itself holds (its repacked weight copies);
 * 0 for a null model.  With gm_workspace_size this gives a step's whole device footprint
 * besides the caller's inputs and outputs. */
GM_API size_t gm_model_device_bytes(const gm_model *m);

/* Bytes of workspace an operation needs (op = GM_OP_*).  nl_capacity is the neighbour
 * list capacity the caller will pass.  Errors: GM_ERR_ARG. */
GM_API gm_status gm_workspace_size(const gm_model *m, int32_t n_structures, int32_t n_atoms,
                            int64_t nl_capacity, int32_t op, size_t *bytes);

/* Neighbour search (cell list, FP32 distance filter with an exact FP64 decision near the
 * cutoff).  Paper: neighbour lists within the cutoff including multiple periodic images
 * for small cells (section "Deployment").  Writes nl->row_ptr, nl->col, nl->shift and
 * *nl->n_pairs.  If more than nl->capacity pairs exist, writes GM_ERR_CAPACITY to
 * *status_dev, the required count to *nl->n_pairs, and leaves col/shift unwritten. */
GM_API gm_status gm_build_neighbors(const gm_model *m, const gm_system *sys, gm_nlist *nl, void *ws,
                             size_t ws_bytes, int32_t *status_dev, struct CUstream_st *stream);

/* Energies and forces (Eqs. energy_sum, basis_fn, contraction, scale_shift; F = -dE/dr).
 *   energy  device [B] FP64, overwritten
 *   forces  device [N][3] FP32, overwritten
 *   virial  device [B][9] FP64 (-dE/d strain, row-major), overwritten; may be NULL
 * The neighbour list must describe sys (as written by gm_build_neighbors or equivalent). */
GM_API gm_status gm_energy_forces(const gm_model *m, const gm_system *sys, const gm_nlist *nl, double *energy,
                           float *forces, double *virial, void *ws, size_t ws_bytes, int32_t *status_dev,
                           struct CUstream_st *stream);

/* ---------------------------------------------------------------- molecular dynamics
 * Section "Deployment": an MD engine whose whole loop runs on the device, with a neighbour
 * list that has a skin and thermostats; the appendix's MD configuration: NVT, dt 0.5 fs, a
 * Nose-Hoover chain (length 3, 2 chain steps, 3 Suzuki-Yoshida steps, tau), skin 0.5 A.
 * Units: A, fs, amu, eV, K. */
typedef enum { GM_MD_NVE = 0, GM_MD_NVT = 1 } gm_md_ensemble;
#define GM_MD_MAX_CHAIN 8

typedef struct {
    double dt;            /* time step (fs) */
    double skin;          /* neighbour-list skin (A): the list holds pairs within r_cut + skin and
                             is rebuilt, on the device, after any atom has moved more than skin/2
                             since the last build */
    double temperature;   /* target temperature (K), NVT */
    double tau;           /* thermostat time constant (fs), NVT: Q_1 = N_f kT tau^2, Q_j = kT tau^2 */
    int32_t ensemble;     /* gm_md_ensemble */
    int32_t chain_length; /* thermostats per chain, 1..GM_MD_MAX_CHAIN (NVT) */
    int32_t chain_steps;  /* sub-steps of each thermostat half step, >= 1 (NVT) */
    int32_t sy_steps;     /* Suzuki-Yoshida stages, 1, 3 or 5 (NVT) */
} gm_md_params;

/* MD state, all device memory owned by the caller (B structures, N atoms, S species). */
typedef struct {
    double *pos;          /* [N][3] positions (A), updated in place; must be sys->pos */
    double *vel;          /* [N][3] velocities (A/fs), in/out */
    const double *mass;   /* [S] masses (amu) */
    float *forces;        /* [N][3] forces at pos (eV/A), written by gm_md_init and every step */
    double *energy;       /* [B] potential energy at pos (eV) */
    double *kinetic;      /* [B] kinetic energy (eV) */
    double *pos_ref;      /* [N][3] positions at the last neighbour build (A) */
    double *chain;        /* [B][2][GM_MD_MAX_CHAIN] thermostat positions xi and velocities v_xi
                             of each structure's chain (NVT; zeroed by gm_md_init) */
    int64_t *n_builds;    /* scalar: neighbour builds, incremented on the device (caller zeroes) */
} gm_md_state;

/* Start (or restart) a run: build the neighbour list at r_cut + skin from state->pos (nl must
 * have room for it), record pos_ref, zero the chains, evaluate forces and energies, the
 * kinetic energies, and count one build.  Workspace: GM_OP_MD with nl's capacity.  Errors:
 * GM_ERR_ARG (null pointers, state->pos != sys->pos, bad parameters), GM_ERR_WORKSPACE. */
GM_API gm_status gm_md_init(const gm_model *m, const gm_system *sys, gm_nlist *nl, const gm_md_params *params,
                            gm_md_state *state, void *ws, size_t ws_bytes, int32_t *status_dev,
                            struct CUstream_st *stream);

/* n_steps steps of velocity Verlet (NVE) or with a Nose-Hoover chain per structure (NVT,
 * integrated with the explicit reversible scheme of Martyna, Tuckerman, Tobias and Klein:
 * a thermostat half step before the first and after the second velocity half kick), with
 * N_f = 3 N_b - 3 degrees of freedom per structure.  Each step: thermostat, half kick and
 * drift, the skin test, the neighbour build only when the test fails (decided on the device),
 * energies and forces, half kick, kinetic energies, thermostat.  Everything is enqueued on
 * `stream` without host synchronisation, so a run can be captured into a CUDA graph and
 * replayed.  A neighbour-list overflow writes GM_ERR_CAPACITY to *status_dev and freezes the
 * state (later kernels skip).  The workspace of gm_md_init; call gm_md_init first. */
GM_API gm_status gm_md_run(const gm_model *m, const gm_system *sys, gm_nlist *nl, const gm_md_params *params,
                           gm_md_state *state, int32_t n_steps, void *ws, size_t ws_bytes, int32_t *status_dev,
                           struct CUstream_st *stream);

/* Force modes of a shallow ensemble (section "Uncertainty Quantification", Eq. jacobian). */
enum { GM_ENS_MEAN_GRADIENT = 0, GM_ENS_JACOBIAN = 1 };

/* Energies and forces of a shallow-ensemble model (desc.n_ensemble = E >= 2 output heads on
 * the last hidden layer; section "Uncertainty Quantification").  Head k gives
 * E_i^(k) = sigma_Zi (w3[:, k] . a2_i + b3[k]) + mu_Zi and E^(k) = sum_i E_i^(k).
 *   energy        device [B] FP64: the mean over heads, Ebar = (1/E) sum_k E^(k)
 *   forces        device [N][3] FP32: -dEbar/dr (Eq. jacobian, left: one backward pass with
 *                 the heads' mean weights)
 *   virial        device [B][9] FP64 of Ebar, or NULL
 *   energy_heads  device [B][E] FP64, E^(k) per structure, or NULL
 *   energy_std    device [B] FP64, sigma_E = sqrt((1/E) sum_k (E^(k) - Ebar)^2) (Eq.
 *                 uncertainty), or NULL
 *   mode          GM_ENS_MEAN_GRADIENT, or GM_ENS_JACOBIAN: also every head's forces
 *                 F^(k) = -dE^(k)/dr (Eq. jacobian, right; E more backward passes), which
 *                 give (with the implied sum over components of Eq. uncertainty)
 *   forces_heads  device [E][N][3] FP32, F^(k), or NULL (GM_ENS_JACOBIAN only)
 *   force_std     device [N] FP32, sigma_F,i = sqrt((1/E) sum_k |F^(k)_i - mean_k F^(k)_i|^2),
 *                 or NULL (GM_ENS_JACOBIAN only)
 * Workspace as GM_OP_ENERGY_FORCES.  gm_energy_forces on an ensemble model returns energy
 * and forces of the mean as above (no per-head outputs).  Errors: GM_ERR_ARG (a model with
 * one head, per-head forces requested in the mean-gradient mode, null or misaligned
 * pointers), GM_ERR_WORKSPACE. */
GM_API gm_status gm_energy_forces_ensemble(const gm_model *m, const gm_system *sys, const gm_nlist *nl,
                                           double *energy, float *forces, double *virial, double *energy_heads,
                                           double *energy_std, int32_t mode, float *forces_heads, float *force_std,
                                           void *ws, size_t ws_bytes, int32_t *status_dev,
                                           struct CUstream_st *stream);

/* Neighbour search that allocates nothing and needs no workspace (the paper has no
 * counterpart; this is a convenience of this library).  Same inputs, outputs, rule and
 * status reporting as gm_build_neighbors, for callers that cannot hand the library
 * device memory: host programs whose own allocator owns all device memory (an MD engine
 * embedding the library), or step loops that must not call cudaMalloc because its
 * implicit synchronisation would stall the other streams mid-step.
 * Scratch is a fixed 8 MiB array in the library's own device memory (a file-scope
 * __device__ variable that every GPU loading the library holds until the process exits),
 * which fits systems whose minimum neighbour workspace, gm_workspace_size(..., nl_capacity
 * = 0, GM_OP_NEIGHBORS), is at most 8 MiB (about 90,000 atoms in one structure; the
 * single-pass search is used when its slab fits too, else the two-pass one).  Larger
 * systems return GM_ERR_WORKSPACE (gm_last_error says why) without launching anything.
 * The arguments are checked as for gm_build_neighbors (GM_ERR_ARG for a null or misaligned
 * pointer), and `stream` must belong to the current device (else GM_ERR_ARG): the cached
 * scratch address is the current device's.
 * The first call on a device, with that device current, looks up the array's device
 * address (cudaGetSymbolAddress) and caches it; make that first call before any stream
 * capture.  All calls share the array and it keeps the last call's contents (the build
 * clears what must start at zero), so calls that overlap on the GPU -- concurrent
 * streams or threads -- race; serialise them. */
GM_API gm_status gm_build_neighbors_noalloc(const gm_model *m, const gm_system *sys, gm_nlist *nl,
                                            int32_t *status_dev, struct CUstream_st *stream);

/* Parameter gradient of a loss through energies and forces (models with one output head;
 * a shallow-ensemble model returns GM_ERR_UNSUPPORTED):
 *   grad_theta = d/dtheta [ sum_b dL_dE[b] E_b + sum_i dL_dF[i] . F_i ]
 * (section "Training": loss terms on energies and forces).  dL_dE device [B] FP64,
 * dL_dF device [N][3] FP32, grad_theta device [gm_param_count] FP32, overwritten.
 * Moments are recomputed from the positions; no per-pair state is stored. */
GM_API gm_status gm_param_grad(const gm_model *m, const gm_system *sys, const gm_nlist *nl, const double *dL_dE,
                        const float *dL_dF, float *grad_theta, void *ws, size_t ws_bytes,
                        int32_t *status_dev, struct CUstream_st *stream);

/* Force-matching loss L = wE/B sum_b ((E_b - E_ref_b)/N_b)^2 + wF/(3N) sum_i |F_i - F_ref_i|^2
 * and its gradients (section "Training": weighted energy and force terms, per-atom
 * division).  loss device scalar FP64; dL_dE device [B] FP64; dL_dF device [N][3] FP32. */
GM_API gm_status gm_force_matching_loss(const gm_system *sys, const double *energy, const double *energy_ref,
                                 const float *forces, const float *forces_ref, double w_energy,
                                 double w_forces, double *loss, double *dL_dE, float *dL_dF,
                                 int32_t *status_dev, struct CUstream_st *stream);

/* Diagnostics: the descriptor of every atom.  psi device [N][n_radial][20] FP32 (unique
 * moment components per radial function: rank 0; x y z; xx xy xz yy yz zz; xxx xxy xxz
 * xyy xyz xzz yyy yyz yzz zzz), features device [N][360] FP32 (may be NULL).
 * Workspace as GM_OP_ENERGY_FORCES. */
GM_API gm_status gm_descriptors(const gm_model *m, const gm_system *sys, const gm_nlist *nl, float *psi,
                         float *features, void *ws, size_t ws_bytes, int32_t *status_dev,
                         struct CUstream_st *stream);

/* Stage timing (the library's built-in tracing).  While enabled, every pipeline stage
 * of gm_build_neighbors / gm_energy_forces / gm_param_grad is bracketed by CUDA events
 * recorded on the call's stream.  gm_profile_collect synchronises those events and
 * returns, per stage, the summed milliseconds and the number of timed occurrences since
 * the last reset, plus the number of kernels the library launched since the last reset
 * (counted whether or not timing is enabled).  Stages are numbered 0..gm_profile_n_stages()-1. */
GM_API void gm_profile_enable(int on);
GM_API void gm_profile_reset(void);
GM_API int gm_profile_n_stages(void);
GM_API const char *gm_profile_stage_name(int stage);
GM_API gm_status gm_profile_collect(double *stage_ms, int64_t *stage_count, int n_stages, int64_t *kernel_launches);
/* Stages recorded while the stream is being captured into a CUDA graph become external
 * event-record nodes of that graph.  gm_profile_collect adds their times again at every
 * call, so call it once after each replay, with the stream synchronised.
 * gm_profile_forget_graphs stops reading them (the events themselves stay allocated, since
 * a graph may still record them). */
GM_API void gm_profile_forget_graphs(void);

/* Throughput probe (no counterpart in the paper; it measures the denominators of the FP32
 * rooflines): launches one kernel of independent chains of a single operation on every SM --
 * kind 0: FP32 fused multiply-add, kind 1: the special-function unit's base-2 exponential --
 * with `iters` iterations of 64 operations per thread, and writes the number of operations
 * launched to *ops (an FMA counts as 2 flop).  Time the launch with CUDA events on `stream`.
 * sink: device float buffer of at least (SMs x 8) entries (never written in practice).
 * Errors: GM_ERR_ARG, GM_ERR_CUDA. */
GM_API gm_status gm_probe_alu(int32_t kind, int64_t iters, float *sink, double *ops, struct CUstream_st *stream);

/* Zero the device status word (cudaMemsetAsync on `stream`); call before each step. */
GM_API gm_status gm_status_clear(int32_t *status_dev, struct CUstream_st *stream);

GM_API const char *gm_status_string(gm_status s);

/* Detail of the last synchronous error on the calling thread ("" if none). */
GM_API const char *gm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GM_H */
