"""The five workload configurations (structures, model sizes, seeds).

    1  4 EMIM+BF4- pairs, 96 atoms, L = 10.09 A; r_c = 5, MLP 2x128 (tanh and SiLU)
    2  64 EMIM+BF4- pairs, 1536 atoms, L = 25.43 A; r_c = 6, MLP 2x512
    3  256 Li3PO4-like structures of 32..512 atoms (multiples of 8), half jittered
       crystal (sigma 0.05 A), half random packing (min sep 1.5 A); r_c = 5, MLP 2x256
    4  32 EMIM+BF4- boxes of 4..16 pairs (96..384 atoms); r_c = 5, MLP 2x128;
       reference energies/forces from a teacher model with its own seed
    5  Li3PO4-like crystal of 16384 formula units, 131072 atoms, L = 109.49 A
       (sigma 0.1 A); r_c = 6, MLP 2x512

Densities: EMIM+BF4- 1.28 g/cm^3, Li3PO4 2.4 g/cm^3.  Mean neighbour counts used to
scale the synthetic species-pair coefficients come from the atom number density.
"""
from __future__ import annotations

import functools
import math

import numpy as np

from .params import make_params
from .systems import (EMIM_SPECIES, LI3PO4_SPECIES, emim_box, emim_pair_mass, box_length,
                      li3po4_crystal, li3po4_random, li3po4_length, make_batch)

EMIM_ATOMS_PER_PAIR = 24


def emim_number_density(density=1.28):
    L = box_length(emim_pair_mass(), density)
    return EMIM_ATOMS_PER_PAIR / L ** 3


def li3po4_number_density(density=2.4):
    return 8.0 / li3po4_length(1, density) ** 3


def mean_neighbours(number_density, r_cut):
    return number_density * 4.0 / 3.0 * math.pi * r_cut ** 3


def model_desc(n_species, n_hidden, r_cut, activation="silu", r_min=0.5, n_basis=7, n_radial=5, basis="gaussian",
               n_ensemble=1):
    return dict(n_species=n_species, n_hidden=n_hidden, r_cut=float(r_cut), r_min=float(r_min),
                n_basis=n_basis, n_radial=n_radial, activation=activation, basis=basis, n_ensemble=n_ensemble)


@functools.lru_cache(maxsize=None)
def _structures(cfg: int):
    if cfg == 1:
        return make_batch([emim_box(4, 1001)], len(EMIM_SPECIES), {"name": "emim-4pairs-96"})
    if cfg == 2:
        return make_batch([emim_box(64, 1002)], len(EMIM_SPECIES), {"name": "emim-64pairs-1536"})
    if cfg == 3:
        rng = np.random.default_rng([1003, 1])
        units = rng.integers(4, 65, size=256)          # 32..512 atoms, multiples of 8
        structs = []
        for b, u in enumerate(units):
            if b % 2 == 0:
                structs.append(li3po4_crystal(int(u), 1003 * 1000 + b, sigma=0.05))
            else:
                structs.append(li3po4_random(int(u), 1003 * 1000 + b, min_sep=1.5))
        return make_batch(structs, len(LI3PO4_SPECIES), {"name": "li3po4-batch-256"})
    if cfg == 4:
        rng = np.random.default_rng([1004, 1])
        pairs = rng.integers(4, 17, size=32)           # 96..384 atoms
        structs = [emim_box(int(p), 1004 * 1000 + b) for b, p in enumerate(pairs)]
        return make_batch(structs, len(EMIM_SPECIES), {"name": "emim-train-32"})
    if cfg == 5:
        return make_batch([li3po4_crystal(16384, 1005, sigma=0.1)], len(LI3PO4_SPECIES),
                          {"name": "li3po4-131072"})
    raise ValueError(cfg)


_MODEL = {
    1: (len(EMIM_SPECIES), 128, 5.0, "emim"),
    2: (len(EMIM_SPECIES), 512, 6.0, "emim"),
    3: (len(LI3PO4_SPECIES), 256, 5.0, "li3po4"),
    4: (len(EMIM_SPECIES), 128, 5.0, "emim"),
    5: (len(LI3PO4_SPECIES), 512, 6.0, "li3po4"),
}

CONFIGS = tuple(_MODEL)


def config(cfg: int, activation="silu", param_seed=None):
    """Return (batch, model_desc, params) for configuration ``cfg``."""
    S, H, rc, kind = _MODEL[cfg]
    batch = _structures(cfg)
    rho = emim_number_density() if kind == "emim" else li3po4_number_density()
    nbar = mean_neighbours(rho, rc)
    desc = model_desc(S, H, rc, activation)
    seed = (cfg + 1000) if param_seed is None else param_seed
    params = make_params(S, H, seed, nbar)
    return batch, desc, params


def teacher_params(cfg: int = 4):
    """Parameters of the random-weight teacher that labels configuration 4."""
    S, H, rc, _ = _MODEL[cfg]
    nbar = mean_neighbours(emim_number_density(), rc)
    return make_params(S, H, 2004, nbar)


def jitter_positions(pos, seed, step, sigma=0.01):
    """Seeded N(0, sigma^2) random-walk increment for MD-like repeated evaluation."""
    rng = np.random.default_rng([seed, 51, step])
    return pos + rng.normal(0.0, sigma, pos.shape)
