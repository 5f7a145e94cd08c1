// gm_md.cu -- molecular dynamics on the device: velocity Verlet, a Nose-Hoover chain per
// structure, and a neighbour list with a skin that is rebuilt only when an atom has moved
// far enough (section "Deployment": the whole simulation loop on the device; the appendix's
// MD configuration: NVT, chain length 3, 2 chain steps, 3 Suzuki-Yoshida steps, tau, skin).
//
// One step, all on the caller's stream (a run of n steps can be captured as one CUDA graph):
//   k_md_kick_drift  v = s v + dt/2 F/m (s: the pending thermostat factor);  r += dt v;
//                    flag if |r - r_ref| > skin / 2
//   neighbour build  at r_cut + skin, gated by the flag (skipped on the device otherwise)
//   energies/forces  the library's pipeline (pairs beyond r_cut contribute exact zeros)
//   k_md_kick_ke     v += dt/2 F/m; r_ref = r after a rebuild; kinetic energy per structure
//                    in fixed point; the last block forms the totals, takes this step's second
//                    thermostat half step and the next step's first (their velocity factor is
//                    applied by the next kick; after the last step of a run only the second,
//                    applied by k_md_finish), clears the flag and counts the build
// k_md_thermo takes the first thermostat half step of a run's first step.
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

// exp(x) - 1 for the thermostat's small arguments: the Taylor series to x^6 / 720 (relative
// error below 2e-9 for |x| < 1/16, under FP32 rounding), expm1f beyond that
__device__ __forceinline__ float em1(float x) {
    if (fabsf(x) < 0.0625f) {
        float p = fmaf(x, 1.0f / 720.0f, 1.0f / 120.0f);
        p = fmaf(x, p, 1.0f / 24.0f);
        p = fmaf(x, p, 1.0f / 6.0f);
        p = fmaf(x, p, 0.5f);
        p = fmaf(x, p, 1.0f);
        return x * p;
    }
    return expm1f(x);
}

// Thermostat half step (dt/2) of one structure with kinetic energy K and N_f degrees of
// freedom; chain = [xi (GM_MD_MAX_CHAIN) | v_xi (GM_MD_MAX_CHAIN)] updated in place.  Returns
// the factor that scales the structure's velocities; *K becomes the scaled kinetic energy.
// One thread runs the whole sequential chain, so its latency is the cost: the chain length M
// is a template parameter (the state lives in registers), the chain's arithmetic is FP32
// (B300's FP64 latency made an FP64 version ~40 us per half step at M = 3 and 2 x 3
// sub-steps), the exponentials of the small arguments are 1 + (e^x - 1) so that 1 - s keeps
// its relative precision, and FP64 appears only before and after the sub-steps (K, the
// increments of the thermostat positions xi).
template <int M>
__device__ double nhc_half_step_m(const MdConst &c, int n_f, double *K, double *chain) {
    double *xi_g = chain, *v_g = chain + GM_MD_MAX_CHAIN;
    const float kT = (float)c.kT;
    const float q0 = (float)((double)n_f * c.kT * c.tau * c.tau), qj = (float)(c.kT * c.tau * c.tau);
    const float iq0 = 1.0f / q0, iqj = 1.0f / qj;
    float v[M], dxi[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
        v[j] = (float)v_g[j];
        dxi[j] = 0.0f;
    }
    float h_sy[5];
#pragma unroll
    for (int a = 0; a < 5; ++a) h_sy[a] = (float)(c.w_sy[a] * c.half_dt / c.chain_steps);
    const double K0 = *K;
    // G_1 = (2K - N_f kT)/Q_1 with K = K0 e^(2X): the difference at X = 0 is formed once in
    // FP64, the change with X in FP32
    const float d0 = (float)(2.0 * K0 - (double)n_f * c.kT), a0 = (float)(2.0 * K0);
    float g0 = d0 * iq0;
    float X = 0.0f;                               // log of the accumulated velocity factor
    auto G = [&](int j) { return j == 0 ? g0 : ((j == 1 ? q0 : qj) * v[j - 1] * v[j - 1] - kT) * iqj; };
    for (int r = 0; r < c.chain_steps; ++r) {
#pragma unroll
        for (int a = 0; a < 5; ++a) {
            if (a >= c.n_sy) break;
            const float h = h_sy[a];
            v[M - 1] += 0.5f * h * G(M - 1);
#pragma unroll
            for (int j = M - 2; j >= 0; --j) {
                const float e = 1.0f + em1(-0.25f * h * v[j + 1]);
                v[j] = (v[j] * e + 0.5f * h * G(j)) * e;
            }
            X -= h * v[0];
            g0 = fmaf(a0, em1(2.0f * X), d0) * iq0;
#pragma unroll
            for (int j = 0; j < M; ++j) dxi[j] = fmaf(h, v[j], dxi[j]);
#pragma unroll
            for (int j = 0; j < M - 1; ++j) {
                const float e = 1.0f + em1(-0.25f * h * v[j + 1]);
                v[j] = (v[j] * e + 0.5f * h * G(j)) * e;
            }
            v[M - 1] += 0.5f * h * G(M - 1);
        }
    }
#pragma unroll
    for (int j = 0; j < M; ++j) {
        v_g[j] = (double)v[j];
        xi_g[j] += (double)dxi[j];
    }
    *K = K0 * (1.0 + (double)em1(2.0f * X));
    return 1.0 + (double)em1(X);
}

__device__ double nhc_half_step(const MdConst &c, int n_f, double *K, double *chain) {
    switch (c.chain_length) {
    case 1: return nhc_half_step_m<1>(c, n_f, K, chain);
    case 2: return nhc_half_step_m<2>(c, n_f, K, chain);
    case 3: return nhc_half_step_m<3>(c, n_f, K, chain);
    case 4: return nhc_half_step_m<4>(c, n_f, K, chain);
    case 5: return nhc_half_step_m<5>(c, n_f, K, chain);
    case 6: return nhc_half_step_m<6>(c, n_f, K, chain);
    case 7: return nhc_half_step_m<7>(c, n_f, K, chain);
    default: return nhc_half_step_m<8>(c, n_f, K, chain);
    }
}

__device__ __forceinline__ int dof_of(const int32_t *atom_ptr, int b) {
    const int n = atom_ptr[b + 1] - atom_ptr[b];
    return n > 1 ? 3 * n - 3 : 3 * n;
}

// First thermostat half step of every structure at the start of a run (later steps take
// theirs in the previous step's k_md_kick_ke); pending[b] = its velocity factor.
__global__ void __launch_bounds__(128) k_md_thermo(int B, const int32_t *__restrict__ atom_ptr, MdConst c,
                                                   double *chain, double *kinetic, double *pending,
                                                   const int32_t *status) {
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
    pending[b] = s;
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
    // acceleration in FP32 (the forces are FP32): no FP64 division on the latency path
    const float inv_m = 1.0f / ((float)mass[species[i]] * (float)AMU_A2_FS2_EV);
    const double s = factor ? factor[structure_of(atom_ptr, B, i)] : 1.0;
    double d2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const size_t q = (size_t)i * 3 + a;
        const double v = s * vel[q] + c.half_dt * (double)(F[q] * inv_m);
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
                                                           int64_t *n_builds, int last_step, const int32_t *status) {
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
        const float inv_m = 1.0f / ((float)m * (float)AMU_A2_FS2_EV);
        double v2 = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const size_t q = (size_t)i * 3 + a;
            double vq = vel[q];
            if (kick) {
                vq += c.half_dt * (double)(F[q] * inv_m);
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
        // this step's second thermostat half step and, unless it is the last step of the run,
        // the next step's first (nothing happens between them): pending is the velocity
        // factor still to apply, by the next kick or by k_md_finish
        for (int s = threadIdx.x; s < B; s += blockDim.x) {
            const int n_f = dof_of(atom_ptr, s);
            double f = 1.0;
            if (n_f > 0) {
                double K = kinetic[s];
                double *ch = chain + (size_t)s * 2 * GM_MD_MAX_CHAIN;
                f = nhc_half_step(c, n_f, &K, ch);
                if (!last_step) f *= nhc_half_step(c, n_f, &K, ch);
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
               double *pending, const int32_t *status, cudaStream_t st) {
    launch_pdl(k_md_thermo, dim3((B + 127) / 128), dim3(128), 0, st, B, atom_ptr, md_const(p), chain, kinetic,
               pending, status);
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
                int last_step, const int32_t *status, cudaStream_t st) {
    const int blocks = N > 0 ? (N + MD_THREADS - 1) / MD_THREADS : 1;
    launch_pdl(k_md_kick_ke, dim3(blocks), dim3(MD_THREADS), 0, st, N, B, atom_ptr, species, mass, F, md_const(p),
               kick, vel, pos, pos_ref, flag, acc, kinetic, chain, pending, n_builds, last_step, status);
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
