"""CPU pins of the FP64 molecular-dynamics reference (oracle.md): velocity Verlet and the
Nose-Hoover chain of Martyna, Tuckerman, Tobias and Klein (section "Deployment" and the MD
configuration of the appendix).

Pinned by: the closed-form discrete trajectory of velocity Verlet on a harmonic oscillator;
conservation of the extended energy H' of the chain (any wrong term, sign or factor in the
thermostat breaks it); time reversibility of the scheme; the chain driving harmonic
oscillators to the target temperature; energy conservation of a short NVE run of the GMNN
oracle model (what the paper's engine integrates), and H' conservation of an NVT run of it.
"""
import math

import numpy as np
import pytest

from oracle import md
from synth.params import make_params, maxwell_boltzmann


def _harmonic(k, x0):
    def fn(pos):
        d = pos - x0
        return np.array([0.5 * (k[:, None] * d * d).sum()]), -k[:, None] * d
    return fn


def test_velocity_verlet_matches_the_closed_form_of_its_discrete_map():
    """x_(n+1) - 2 cos(theta) x_n + x_(n-1) = 0 with cos(theta) = 1 - (w dt)^2 / 2, so
    x_n = x_0 cos(n theta) + dt v_0 sin(n theta) / sin(theta)."""
    m = np.array([6.94])
    k = np.array([2.3])                       # eV/A^2
    x0 = np.zeros((1, 3))
    pos = np.array([[0.3, -0.1, 0.05]])
    vel = np.array([[0.004, 0.01, -0.002]])   # A/fs
    dt, n = 0.5, 1000
    w2 = k[0] / (m[0] * md.AMU_A2_PER_FS2_IN_EV)
    theta = math.acos(1.0 - 0.5 * w2 * dt * dt)
    p, v, _, _, _ = md.integrate(pos, vel, m, np.array([0, 1]), _harmonic(k, x0), dt, n)
    want = pos * math.cos(n * theta) + dt * vel * math.sin(n * theta) / math.sin(theta)
    assert np.allclose(p, want, rtol=0, atol=1e-12)


NVT = {"temperature": 600.0, "tau": 50.0, "chain_length": 3, "chain_steps": 2, "sy_steps": 3}


def _oscillators(n=64, seed=3):
    rng = np.random.default_rng(seed)
    m = rng.choice([6.94, 30.974, 15.999], n)
    k = rng.uniform(0.5, 4.0, n)
    x0 = rng.uniform(0, 10, (n, 3))
    pos = x0 + rng.normal(0, 0.05, (n, 3))
    vel = maxwell_boltzmann(m, np.array([0, n]), 300.0, seed)
    return m, k, x0, pos, vel


def _extended_energy(pos, vel, m, fn, chains, ap):
    E, _ = fn(pos)
    return E[0] + md.kinetic(vel, m, ap)[0] + chains[0].energy()


def test_nose_hoover_chain_conserves_the_extended_energy_and_thermostats():
    m, k, x0, pos, vel = _oscillators()
    ap = np.array([0, len(m)])
    fn = _harmonic(k, x0)
    p, v, _, _, ch = md.integrate(pos, vel, m, ap, fn, 0.5, 200, nvt=NVT)
    h0 = _extended_energy(p, v, m, fn, ch, ap)
    kT = md.KB_EV_PER_K * NVT["temperature"]
    temps, hs = [], []
    for _ in range(60):
        p, v, _, _, ch = md.integrate(p, v, m, ap, fn, 0.5, 100, nvt=NVT, chains=ch)
        hs.append(_extended_energy(p, v, m, fn, ch, ap))
        temps.append(2 * md.kinetic(v, m, ap)[0] / (md.degrees_of_freedom(len(m)) * md.KB_EV_PER_K))
    # H' stays within 1e-4 N_f kT over 6000 steps (the size of velocity Verlet's own energy
    # fluctuation at (w dt)^2 ~ 1e-3), while the kinetic energy changes by about N_f kT / 2 as
    # the chain heats the oscillators from 300 to 600 K
    n_f = md.degrees_of_freedom(len(m))
    assert max(abs(h - h0) for h in hs) < 1e-4 * n_f * kT
    assert abs(np.mean(temps[20:]) - NVT["temperature"]) < 0.1 * NVT["temperature"]


def test_nose_hoover_chain_is_time_reversible():
    m, k, x0, pos, vel = _oscillators(16, 5)
    ap = np.array([0, len(m)])
    fn = _harmonic(k, x0)
    p, v, _, _, ch = md.integrate(pos, vel, m, ap, fn, 0.5, 50, nvt=NVT)
    for c in ch:
        c.v = -c.v
    p2, v2, _, _, ch2 = md.integrate(p, -v, m, ap, fn, 0.5, 50, nvt=NVT, chains=ch)
    assert np.allclose(p2, pos, atol=1e-10) and np.allclose(-v2, vel, atol=1e-12)
    assert np.allclose(ch2[0].xi, 0.0, atol=1e-10) and np.allclose(ch2[0].v, 0.0, atol=1e-12)


@pytest.fixture(scope="module")
def li192():
    import synth
    from synth.systems import li3po4_crystal, make_batch, species_masses
    _, d, p = synth.config(3)
    b = make_batch([li3po4_crystal(24, 777, sigma=0.05)], 3)
    masses = species_masses("li3po4")[b.species]
    vel = maxwell_boltzmann(masses, b.atom_ptr, 600.0, 11)
    return b, d, p, masses, vel


def test_gmnn_nve_conserves_energy(li192):
    b, d, p, masses, vel = li192
    fn = md.gmnn_force_fn(b, d, p)
    E0, _ = fn(b.pos)
    tot0 = E0[0] + md.kinetic(vel, masses, b.atom_ptr)[0]
    pos, v, E, _, _ = md.integrate(b.pos, vel, masses, b.atom_ptr, fn, 0.5, 100)
    tot = E[0] + md.kinetic(v, masses, b.atom_ptr)[0]
    kT = md.KB_EV_PER_K * 600.0
    assert abs(tot - tot0) < 1e-4 * kT * b.n_atoms
    assert np.abs(pos - b.pos).max() > 0.05                  # the atoms did move


def test_gmnn_nvt_conserves_the_extended_energy(li192):
    b, d, p, masses, vel = li192
    fn = md.gmnn_force_fn(b, d, p)
    nvt = dict(NVT, tau=5.0)                                  # a strongly coupled chain
    pos, v, E, _, ch = md.integrate(b.pos, vel, masses, b.atom_ptr, fn, 0.5, 10, nvt=nvt)
    h0 = E[0] + md.kinetic(v, masses, b.atom_ptr)[0] + ch[0].energy()
    pos, v, E, _, ch = md.integrate(pos, v, masses, b.atom_ptr, fn, 0.5, 60, nvt=nvt, chains=ch)
    h1 = E[0] + md.kinetic(v, masses, b.atom_ptr)[0] + ch[0].energy()
    kT = md.KB_EV_PER_K * 600.0
    assert abs(h1 - h0) < 1e-4 * kT * b.n_atoms
    assert abs(ch[0].v).max() > 0                             # the thermostat acted
