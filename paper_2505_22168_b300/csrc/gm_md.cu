// gm_md.cu -- molecular dynamics on the device: velocity Verlet, a Nose-Hoover chain per
// structure, and a neighbour list with a skin that is rebuilt only when an atom has moved
// far enough (section "Deployment": the whole simulation loop on the device; the appendix's
// MD configuration: NVT, chain length 3, 2 chain steps, 3 Suzuki-Yoshida steps, tau, skin).
//
// One step, all on the caller's stream (a run of n steps can be captured as one CUDA graph):
//   k_md_thermo      NVT: first thermostat half step of every structure (one thread each)
//   k_md_kick_drift  v = s v + dt/2 F/m;  r += dt v;  flag if |r - r_ref| > skin / 2
//   neighbour build  at r_cut + skin, gated by the flag (skipped on the device otherwise)
//   energies/forces  the library's pipeline (pairs beyond r_cut contribute exact zeros)
//   k_md_kick_ke     v += dt/2 F/m; r_ref = r after a rebuild; kinetic energy per structure
//                    in fixed point; the last block forms the totals, takes the second
//                    thermostat half step (its velocity factor is applied by the next kick, or
//                    by k_md_finish after the last step), clears the flag and counts the build
// The thermostat integrates the chain equations of motion with the explicit reversible
// Trotter scheme of Martyna, Tuckerman, Tobias and Klein (1996): chain_steps x Suzuki-Yoshida
// sub-steps per half step, masses Q_1 = N_f kT tau^2 and Q_j = kT tau^2, N_f = 3 N_b - 3.
#include <math.h>

#include "gm_fixed.cuh"
#include "gm_md.h"

namespace gm {

constexpr double AMU_A2_FS2_EV = 103.642696562;   // 1 amu A^2 / fs^2 in eV
constexpr double KB_EV = 8.617333262e-5;           // eV / K
constexpr int MD_THREADS = 256;

struct MdConst {
    double dt, half_dt, skin_half2, kT, tau;
    int nvt, chain_length, chain_steps, n_sy;
    double w_sy[5];
};

MdConst md_const(const gm_md_params &p) {
    MdConst c;
    c.dt = p.dt;
    c.half_dt = 0.5 * p.dt;
    c.skin_half2 = 0.25 * p.skin * p.skin;
    c.kT = KB_EV * p.temperature;
    c.tau = p.tau;
    c.nvt = p.ensemble == GM_MD_NVT ? 1 : 0;
    c.chain_length = p.chain_length;
    c.chain_steps = p.chain_steps;
    c.n_sy = p.sy_steps;
    for (int i = 0; i < 5; ++i) c.w_sy[i] = 0.0;
    if (p.sy_steps == 1) {
        c.w_sy[0] = 1.0;
    } else if (p.sy_steps == 3) {       // fourth-order Suzuki-Yoshida weights
        const double w = 1.0 / (2.0 - cbrt(2.0));
        c.w_sy[0] = c.w_sy[2] = w;
        c.w_sy[1] = 1.0 - 2.0 * w;
    } else {
        const double w = 1.0 / (4.0 - cbrt(4.0));
        c.w_sy[0] = c.w_sy[1] = c.w_sy[3] = c.w_sy[4] = w;
        c.w_sy[2] = 1.0 - 4.0 * w;
    }
    return c;
}

// Thermostat half step (dt/2) of one structure with kinetic energy K and N_f degrees of
// freedom; chain = [xi (GM_MD_MAX_CHAIN) | v_xi (GM_MD_MAX_CHAIN)] updated in place.  Returns
// the factor that scales the structure's velocities; *K becomes the scaled kinetic energy.
__device__ double nhc_half_step(const MdConst &c, int n_f, double *K, double *chain) {
    const int M = c.chain_length;
    double *xi = chain, *v = chain + GM_MD_MAX_CHAIN;
    const double q0 = (double)n_f * c.kT * c.tau * c.tau, qj = c.kT * c.tau * c.tau;
    auto Q = [&](int j) { return j == 0 ? q0 : qj; };
    auto G = [&](int j, double kin) {
        return j == 0 ? (2.0 * kin - (double)n_f * c.kT) / q0 : (Q(j - 1) * v[j - 1] * v[j - 1] - c.kT) / qj;
    };
    double kin = *K, scale = 1.0;
    for (int r = 0; r < c.chain_steps; ++r) {
        for (int a = 0; a < c.n_sy; ++a) {
            const double h = c.w_sy[a] * c.half_dt / c.chain_steps;
            v[M - 1] += 0.5 * h * G(M - 1, kin);
            for (int j = M - 2; j >= 0; --j) {
                const double e = exp(-0.25 * h * v[j + 1]);
                v[j] = (v[j] * e + 0.5 * h * G(j, kin)) * e;
            }
            const double s = exp(-h * v[0]);
            scale *= s;
            kin *= s * s;
            for (int j = 0; j < M; ++j) xi[j] += h * v[j];
            for (int j = 0; j < M - 1; ++j) {
                const double e = exp(-0.25 * h * v[j + 1]);
                v[j] = (v[j] * e + 0.5 * h * G(j, kin)) * e;
            }
            v[M - 1] += 0.5 * h * G(M - 1, kin);
        }
    }
    *K = kin;
    return scale;
}

__device__ __forceinline__ int dof_of(const int32_t *atom_ptr, int b) {
    const int n = atom_ptr[b + 1] - atom_ptr[b];
    return n > 1 ? 3 * n - 3 : 3 * n;
}

// First thermostat half step of every structure; factor[b] = (pending from the previous
// step's second half, unless first) x this half step's factor.
__global__ void __launch_bounds__(128) k_md_thermo(int B, const int32_t *__restrict__ atom_ptr, MdConst c,
                                                   double *chain, double *kinetic, const double *pending,
                                                   double *factor, int first, const int32_t *status) {
    griddep_wait();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B || status_bad(status)) return;
    const int n_f = dof_of(atom_ptr, b);
    double s = 1.0;
    if (n_f > 0) {
        double K = kinetic[b];
        s = nhc_half_step(c, n_f, &K, chain + (size_t)b * 2 * GM_MD_MAX_CHAIN);
        kinetic[b] = K;
    }
    factor[b] = first ? s : pending[b] * s;
}

// v = s_b v + dt/2 F/m;  r += dt v;  the skin test against the positions of the last build
__global__ void __launch_bounds__(MD_THREADS) k_md_kick_drift(int N, int B, const int32_t *__restrict__ atom_ptr,
                                                              const int32_t *__restrict__ species,
                                                              const double *__restrict__ mass,
                                                              const float *__restrict__ F, const double *factor,
                                                              MdConst c, double *vel, double *pos,
                                                              const double *__restrict__ pos_ref, int32_t *flag,
                                                              const int32_t *status) {
    griddep_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N || status_bad(status)) return;
    const double inv_m = 1.0 / (mass[species[i]] * AMU_A2_FS2_EV);
    const double s = factor ? factor[structure_of(atom_ptr, B, i)] : 1.0;
    double d2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const size_t q = (size_t)i * 3 + a;
        const double v = s * vel[q] + c.half_dt * (double)F[q] * inv_m;
        const double x = pos[q] + c.dt * v;
        vel[q] = v;
        pos[q] = x;
        const double d = x - pos_ref[q];
        d2 += d * d;
    }
    if (d2 > c.skin_half2) *reinterpret_cast<volatile int32_t *>(flag) = 1;
}

// v += dt/2 F/m (kick = 1); r_ref = r after a rebuild; kinetic energy per structure.  The
// last block: kinetic totals, the second thermostat half step (factor to pending), flag
// cleared and the build counted.
__global__ void __launch_bounds__(MD_THREADS) k_md_kick_ke(int N, int B, const int32_t *__restrict__ atom_ptr,
                                                           const int32_t *__restrict__ species,
                                                           const double *__restrict__ mass,
                                                           const float *__restrict__ F, MdConst c, int kick,
                                                           double *vel, const double *__restrict__ pos,
                                                           double *pos_ref, int32_t *flag, unsigned long long *acc,
                                                           double *kinetic, double *chain, double *pending,
                                                           int64_t *n_builds, const int32_t *status) {
    __shared__ bool last;
    griddep_wait();
    if (status_bad(status)) return;                    // every block: no ticket, nothing added
    const int i = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31;
    const bool rebuilt = *reinterpret_cast<const volatile int32_t *>(flag) != 0;
    long long v[1] = {0};
    int b = -1;
    bool bad = false;
    if (i < N) {
        const double m = mass[species[i]];
        const double inv_m = 1.0 / (m * AMU_A2_FS2_EV);
        double v2 = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const size_t q = (size_t)i * 3 + a;
            double vq = vel[q];
            if (kick) {
                vq += c.half_dt * (double)F[q] * inv_m;
                vel[q] = vq;
            }
            if (rebuilt) pos_ref[q] = pos[q];
            v2 += vq * vq;
        }
        v[0] = to_fixed((float)(0.5 * AMU_A2_FS2_EV * m * v2), bad);
        b = structure_of(atom_ptr, B, i);
    }
    warp_add_fixed<1>(b, v, 1, bad, acc, lane);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long ticket = atomicAdd(acc + (size_t)B * RW, 1ull);
        last = ticket == (unsigned long long)(gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    finalize_fixed(B, 1, acc, kinetic, nullptr, threadIdx.x, blockDim.x, [] { __syncthreads(); });
    __syncthreads();
    __threadfence();
    if (c.nvt) {
        for (int s = threadIdx.x; s < B; s += blockDim.x) {
            const int n_f = dof_of(atom_ptr, s);
            double f = 1.0;
            if (n_f > 0) {
                double K = kinetic[s];
                f = nhc_half_step(c, n_f, &K, chain + (size_t)s * 2 * GM_MD_MAX_CHAIN);
                kinetic[s] = K;
            }
            pending[s] = f;
        }
    }
    if (threadIdx.x == 0 && rebuilt) {
        *flag = 0;
        if (n_builds) *n_builds += 1;
    }
}

// after the last step: the second thermostat half step's velocity factor
__global__ void __launch_bounds__(MD_THREADS) k_md_finish(int N, int B, const int32_t *__restrict__ atom_ptr,
                                                          const double *pending, double *vel, const int32_t *status) {
    griddep_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N || status_bad(status)) return;
    const double s = pending[structure_of(atom_ptr, B, i)];
#pragma unroll
    for (int a = 0; a < 3; ++a) vel[(size_t)i * 3 + a] *= s;
}

// ------------------------------------------------------------------------------ host side

gm_status md_check_params(const gm_md_params *p) {
    if (!p) return GM_ERR_ARG;
    if (!(p->dt > 0.0) || !(p->skin >= 0.0)) return GM_ERR_ARG;
    if (p->ensemble != GM_MD_NVE && p->ensemble != GM_MD_NVT) return GM_ERR_ARG;
    if (p->ensemble == GM_MD_NVT) {
        if (!(p->temperature > 0.0) || !(p->tau > 0.0)) return GM_ERR_ARG;
        if (p->chain_length < 1 || p->chain_length > GM_MD_MAX_CHAIN || p->chain_steps < 1) return GM_ERR_ARG;
        if (p->sy_steps != 1 && p->sy_steps != 3 && p->sy_steps != 5) return GM_ERR_ARG;
    }
    return GM_OK;
}

void md_thermo(int B, const int32_t *atom_ptr, const gm_md_params &p, double *chain, double *kinetic,
               const double *pending, double *factor, int first, const int32_t *status, cudaStream_t st) {
    launch_pdl(k_md_thermo, dim3((B + 127) / 128), dim3(128), 0, st, B, atom_ptr, md_const(p), chain, kinetic,
               pending, factor, first, status);
    note_launches(1);
}

void md_kick_drift(int N, int B, const int32_t *atom_ptr, const int32_t *species, const double *mass, const float *F,
                   const double *factor, const gm_md_params &p, double *vel, double *pos, const double *pos_ref,
                   int32_t *flag, const int32_t *status, cudaStream_t st) {
    if (N <= 0) return;
    launch_pdl(k_md_kick_drift, dim3((N + MD_THREADS - 1) / MD_THREADS), dim3(MD_THREADS), 0, st, N, B, atom_ptr,
               species, mass, F, factor, md_const(p), vel, pos, pos_ref, flag, status);
    note_launches(1);
}

void md_kick_ke(int N, int B, const int32_t *atom_ptr, const int32_t *species, const double *mass, const float *F,
                const gm_md_params &p, int kick, double *vel, const double *pos, double *pos_ref, int32_t *flag,
                unsigned long long *acc, double *kinetic, double *chain, double *pending, int64_t *n_builds,
                const int32_t *status, cudaStream_t st) {
    const int blocks = N > 0 ? (N + MD_THREADS - 1) / MD_THREADS : 1;
    launch_pdl(k_md_kick_ke, dim3(blocks), dim3(MD_THREADS), 0, st, N, B, atom_ptr, species, mass, F, md_const(p),
               kick, vel, pos, pos_ref, flag, acc, kinetic, chain, pending, n_builds, status);
    note_launches(1);
}

void md_finish(int N, int B, const int32_t *atom_ptr, const double *pending, double *vel, const int32_t *status,
               cudaStream_t st) {
    if (N <= 0) return;
    launch_pdl(k_md_finish, dim3((N + MD_THREADS - 1) / MD_THREADS), dim3(MD_THREADS), 0, st, N, B, atom_ptr, pending,
               vel, status);
    note_launches(1);
}

}  // namespace gm
