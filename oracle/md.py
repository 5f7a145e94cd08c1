"""FP64 reference of the molecular-dynamics loop.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU
legs use this module; the GPU library never does, and it never imports the GPU library.

Section "Deployment" of the paper: an MD engine whose whole simulation loop runs on the
device, with thermostats and a neighbour list with a skin; the MD configuration in the
appendix ("Input file for performing a JAX-based MD simulation"): NVT, a 0.5 fs time step,
a Nose-Hoover chain of length 3 with 2 chain steps and 3 Suzuki-Yoshida steps and time
constant 100, and a neighbour-list skin (dr_threshold) of 0.5 A.  The time per MD step of
Table li3po4_perf covers this whole loop.

What is computed here, per structure b with N_f = 3 N_b - 3 degrees of freedom (3 for a
single atom), in eV, A, fs and amu:
  velocity Verlet   v += dt/2 F/m;  r += dt v;  F = F(r);  v += dt/2 F/m
  NVT               the Nose-Hoover chain equations of motion
                      dv/dt      = F/m - v_xi1 v
                      dxi_j/dt   = v_xij
                      dv_xi1/dt  = (2K - N_f kT)/Q_1 - v_xi1 v_xi2
                      dv_xij/dt  = (Q_(j-1) v_xi(j-1)^2 - kT)/Q_j - v_xij v_xi(j+1)
                      dv_xiM/dt  = (Q_(M-1) v_xi(M-1)^2 - kT)/Q_M
                    with Q_1 = N_f kT tau^2, Q_j = kT tau^2, integrated by the explicit
                    reversible scheme of Martyna, Tuckerman, Tobias and Klein (1996): a thermostat
                    half step before the first and after the second velocity half kick, each
                    made of chain_steps x (Suzuki-Yoshida weights) symmetric Trotter sub-steps;
                    it conserves H' = K + U + sum_j Q_j v_xij^2 / 2 + N_f kT xi_1 + kT sum_(j>1) xi_j
  forces            recomputed from scratch each step (brute-force neighbour list at r_cut and
                    the oracle's energy and forces): the skin of the GPU list is an
                    optimisation that must not change the result beyond rounding.
Readings: tau is in units of the time step (tau = 100 dt for the appendix configuration);
N_f excludes the centre-of-mass motion.
"""
from __future__ import annotations

import math

import numpy as np

AMU_A2_PER_FS2_IN_EV = 103.642696562      # 1 amu A^2 / fs^2 in eV (CODATA amu and eV)
KB_EV_PER_K = 8.617333262e-5               # Boltzmann constant in eV/K


def suzuki_yoshida_weights(n: int):
    """Weights of the fourth-order Suzuki-Yoshida factorisation with n = 1, 3 or 5 stages."""
    if n == 1:
        return [1.0]
    if n == 3:
        w = 1.0 / (2.0 - 2.0 ** (1.0 / 3.0))
        return [w, 1.0 - 2.0 * w, w]
    if n == 5:
        w = 1.0 / (4.0 - 4.0 ** (1.0 / 3.0))
        return [w, w, 1.0 - 4.0 * w, w, w]
    raise ValueError("Suzuki-Yoshida steps must be 1, 3 or 5")


def degrees_of_freedom(n_atoms: int) -> int:
    return 3 * n_atoms - 3 if n_atoms > 1 else 3


class Chain:
    """Nose-Hoover chain of one structure: positions xi and velocities v_xi of M thermostats."""

    def __init__(self, length, n_f, kT, tau):
        self.M, self.n_f, self.kT = length, n_f, kT
        self.Q = np.array([n_f * kT * tau * tau] + [kT * tau * tau] * (length - 1))
        self.xi = np.zeros(length)
        self.v = np.zeros(length)

    def energy(self):
        """Thermostat part of the conserved quantity."""
        return 0.5 * (self.Q * self.v ** 2).sum() + self.n_f * self.kT * self.xi[0] + self.kT * self.xi[1:].sum()

    def _G(self, j, K):
        if j == 0:
            return (2.0 * K - self.n_f * self.kT) / self.Q[0]
        return (self.Q[j - 1] * self.v[j - 1] ** 2 - self.kT) / self.Q[j]

    def half_step(self, K, dt, chain_steps, weights):
        """Apply the thermostat for dt/2 given the kinetic energy K; returns the factor that
        scales every velocity of the structure (the kinetic energy scales by its square)."""
        M = self.M
        scale = 1.0
        for _ in range(chain_steps):
            for w in weights:
                h = w * 0.5 * dt / chain_steps          # one symmetric sub-step of length h
                self.v[M - 1] += 0.5 * h * self._G(M - 1, K)
                for j in range(M - 2, -1, -1):
                    e = math.exp(-0.25 * h * self.v[j + 1])
                    self.v[j] = (self.v[j] * e + 0.5 * h * self._G(j, K)) * e
                s = math.exp(-h * self.v[0])
                scale *= s
                K *= s * s
                self.xi += h * self.v
                for j in range(M - 1):
                    e = math.exp(-0.25 * h * self.v[j + 1])
                    self.v[j] = (self.v[j] * e + 0.5 * h * self._G(j, K)) * e
                self.v[M - 1] += 0.5 * h * self._G(M - 1, K)
        return scale


def kinetic(vel, m_atom, atom_ptr):
    """Kinetic energy per structure (eV)."""
    ke = 0.5 * AMU_A2_PER_FS2_IN_EV * m_atom * (vel ** 2).sum(1)
    return np.array([ke[atom_ptr[b]:atom_ptr[b + 1]].sum() for b in range(len(atom_ptr) - 1)])


def integrate(pos, vel, m_atom, atom_ptr, force_fn, dt, n_steps, nvt=None, chains=None):
    """Velocity Verlet (optionally with the Nose-Hoover chain of every structure) for n_steps.

    force_fn(pos) -> (E [B], F [N, 3]) in eV and eV/A; m_atom [N] amu; nvt: dict with
    temperature (K), tau (fs), chain_length, chain_steps, sy_steps.  chains: the structures'
    Chain objects (created at zero when None).  Returns (pos, vel, E, F, chains), all updated."""
    pos = np.array(pos, np.float64)
    vel = np.array(vel, np.float64)
    B = len(atom_ptr) - 1
    sid = np.repeat(np.arange(B), np.diff(atom_ptr))
    inv_m = 1.0 / (m_atom * AMU_A2_PER_FS2_IN_EV)
    E, F = force_fn(pos)
    weights = None
    if nvt is not None:
        kT = KB_EV_PER_K * nvt["temperature"]
        weights = suzuki_yoshida_weights(nvt["sy_steps"])
        if chains is None:
            chains = [Chain(nvt["chain_length"], degrees_of_freedom(atom_ptr[b + 1] - atom_ptr[b]), kT, nvt["tau"])
                      for b in range(B)]
    for _ in range(n_steps):
        if nvt is not None:
            K = kinetic(vel, m_atom, atom_ptr)
            s = np.array([chains[b].half_step(K[b], dt, nvt["chain_steps"], weights) for b in range(B)])
            vel *= s[sid][:, None]
        vel += 0.5 * dt * F * inv_m[:, None]
        pos += dt * vel
        E, F = force_fn(pos)
        vel += 0.5 * dt * F * inv_m[:, None]
        if nvt is not None:
            K = kinetic(vel, m_atom, atom_ptr)
            s = np.array([chains[b].half_step(K[b], dt, nvt["chain_steps"], weights) for b in range(B)])
            vel *= s[sid][:, None]
    return pos, vel, E, F, chains


def gmnn_force_fn(batch, desc, params):
    """Forces of the FP64 oracle model at given positions (fresh brute-force list each call)."""
    import dataclasses

    from . import energy_forces, neighbors

    def fn(pos):
        b = dataclasses.replace(batch, pos=pos) if dataclasses.is_dataclass(batch) else batch
        nl = neighbors(b, desc["r_cut"])
        out = energy_forces(b, desc, params, nl, virial=False)
        return out["E"], out["F"]
    return fn
