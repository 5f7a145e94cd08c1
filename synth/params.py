"""Seeded synthetic GMNN parameters (no trained weights exist here).

Only random draws happen here: shapes follow the model (species-pair coefficients,
two hidden layers, linear output, per-species scale and shift), scales follow common
initialisations.  Returned as a dict of named float64 arrays; each side (oracle, GPU
binding) packs them its own way.

    beta  [S, S, n_radial, n_basis]  ~ N(0, (24 / nbar)^2)   (rank-0 moments ~ O(1),
                                     so that all eight contraction families contribute)
    W1    [n_features, H]            Xavier normal
    b1    [H]                        ~ N(0, 0.1^2)
    W2    [H, H]                     Xavier normal
    b2    [H]                        ~ N(0, 0.1^2)
    w3    [H] (or [H, E] for E heads) Xavier normal (fan_out 1 per head)
    b3    [1] (or [E])               ~ N(0, 0.1^2)
    sigma [S]                        ~ U(0.5, 1.5)
    mu    [S]                        ~ N(0, 1)
"""
from __future__ import annotations

import math

import numpy as np

N_FEATURES = 360
BETA_SCALE = 24.0


def param_shapes(n_species: int, n_hidden: int, n_radial=5, n_basis=7, n_features=N_FEATURES, n_ensemble=1):
    """Parameter shapes; a shallow ensemble of E > 1 output heads has w3 [H, E] and b3 [E]."""
    S, H, E = n_species, n_hidden, max(1, int(n_ensemble))
    return {
        "beta": (S, S, n_radial, n_basis),
        "W1": (n_features, H),
        "b1": (H,),
        "W2": (H, H),
        "b2": (H,),
        "w3": (H,) if E == 1 else (H, E),
        "b3": (E,),
        "sigma": (S,),
        "mu": (S,),
    }


def make_params(n_species: int, n_hidden: int, seed: int, nbar: float,
                n_radial=5, n_basis=7, n_features=N_FEATURES, n_ensemble=1):
    rng = np.random.default_rng([seed, 41])
    sh = param_shapes(n_species, n_hidden, n_radial, n_basis, n_features, n_ensemble)

    def xavier(fan_in, fan_out, shape):
        return rng.normal(0.0, math.sqrt(2.0 / (fan_in + fan_out)), shape)

    H = n_hidden
    p = {
        "beta": rng.normal(0.0, BETA_SCALE / nbar, sh["beta"]),
        "W1": xavier(n_features, H, sh["W1"]),
        "b1": rng.normal(0.0, 0.1, sh["b1"]),
        "W2": xavier(H, H, sh["W2"]),
        "b2": rng.normal(0.0, 0.1, sh["b2"]),
        "w3": xavier(H, 1, sh["w3"]),
        "b3": rng.normal(0.0, 0.1, sh["b3"]),
        "sigma": rng.uniform(0.5, 1.5, sh["sigma"]),
        "mu": rng.normal(0.0, 1.0, sh["mu"]),
    }
    return {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in p.items()}


def maxwell_boltzmann(masses_amu, atom_ptr, temperature_k, seed):
    """Seeded initial velocities (A/fs): each component ~ N(0, kT/m), then every structure's
    centre-of-mass velocity removed.  Input generation only (the MD integrators on both sides
    take these as given)."""
    kb, conv = 8.617333262e-5, 103.642696562      # eV/K; amu A^2/fs^2 in eV
    rng = np.random.default_rng([seed, 61])
    m = np.asarray(masses_amu, np.float64)
    v = rng.normal(0.0, 1.0, (len(m), 3)) * np.sqrt(kb * temperature_k / (m * conv))[:, None]
    for b in range(len(atom_ptr) - 1):
        a0, a1 = atom_ptr[b], atom_ptr[b + 1]
        if a1 - a0 > 1:
            v[a0:a1] -= (m[a0:a1, None] * v[a0:a1]).sum(0) / m[a0:a1].sum()
    return v
