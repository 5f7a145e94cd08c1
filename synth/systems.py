"""Seeded synthetic atomic systems (positions, species, periodic cells).

The paper's performance workloads are an EMIM+BF4- ionic liquid (Results, "Inference
Performance") and the Li3PO4 solid electrolyte (Table li3po4_perf).  Neither dataset is
available here, so these generators build stand-ins with the same composition, density,
atom counts and neighbour counts:

* EMIM+BF4-: approximate molecular templates (ring and substituents from standard bond
  lengths; tetrahedral BF4-) at seeded random orientations on a jittered grid, rejecting
  placements that bring atoms of different molecules closer than ``min_sep``.
* Li3PO4: either a jittered "crystal" (a simple cubic site lattice carrying a 2x2x2
  motif of 1 P, 4 O and 3 Li; surplus sites are left vacant at random) or a random
  packing with a hard minimum separation.

All lengths are in Angstrom.  Cells are cubic; rows of ``cell`` are lattice vectors.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

AVOGADRO = 6.02214076e23

# Species indices used by the generators (index into per-species model parameters).
EMIM_SPECIES = {"H": 0, "C": 1, "N": 2, "B": 3, "F": 4}
LI3PO4_SPECIES = {"Li": 0, "P": 1, "O": 2}

_MASS = {"H": 1.008, "C": 12.011, "N": 14.007, "B": 10.81, "F": 18.998,
         "Li": 6.94, "P": 30.974, "O": 15.999}


@dataclass
class Batch:
    """A batch of periodic structures laid out as one ragged array of atoms.

    pos      float64 [N, 3]   Cartesian positions
    species  int32   [N]      species index, 0 <= s < n_species
    atom_ptr int32   [B + 1]  structure b owns atoms atom_ptr[b] .. atom_ptr[b+1]-1
    cell     float64 [B, 3, 3] rows are lattice vectors
    pbc      uint8   [B, 3]   periodic flags per axis
    """
    pos: np.ndarray
    species: np.ndarray
    atom_ptr: np.ndarray
    cell: np.ndarray
    pbc: np.ndarray
    n_species: int
    meta: dict = field(default_factory=dict)

    @property
    def n_atoms(self) -> int:
        return int(self.atom_ptr[-1])

    @property
    def n_structures(self) -> int:
        return int(len(self.atom_ptr) - 1)

    def counts(self) -> np.ndarray:
        return np.diff(self.atom_ptr)


def make_batch(structures, n_species, meta=None) -> Batch:
    """Concatenate a list of (pos, species, cell) tuples into a Batch (all periodic)."""
    pos = np.concatenate([np.asarray(s[0], np.float64).reshape(-1, 3) for s in structures])
    spec = np.concatenate([np.asarray(s[1], np.int32) for s in structures])
    counts = [len(s[1]) for s in structures]
    atom_ptr = np.zeros(len(structures) + 1, np.int32)
    atom_ptr[1:] = np.cumsum(counts)
    cell = np.stack([np.asarray(s[2], np.float64) for s in structures])
    pbc = np.ones((len(structures), 3), np.uint8)
    return Batch(np.ascontiguousarray(pos), np.ascontiguousarray(spec), atom_ptr,
                 np.ascontiguousarray(cell), pbc, n_species, dict(meta or {}))


def box_length(total_mass_amu: float, density_g_cm3: float) -> float:
    """Edge of the cube holding ``total_mass_amu`` at ``density_g_cm3`` (Angstrom)."""
    volume_cm3 = total_mass_amu / AVOGADRO / density_g_cm3
    return (volume_cm3 * 1e24) ** (1.0 / 3.0)


# --------------------------------------------------------------------------- EMIM+BF4-

def _perp_basis(a):
    a = a / np.linalg.norm(a)
    t = np.array([1.0, 0.0, 0.0]) if abs(a[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(a, t)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(a, e1)
    return a, e1, e2


def _tetra_arm(parent, center, phi, length):
    """Point at ``length`` from ``center``, 109.47 deg from the center->parent bond."""
    a, e1, e2 = _perp_basis(center - parent)
    th = math.radians(180.0 - 109.47)
    d = math.cos(th) * a + math.sin(th) * (math.cos(phi) * e1 + math.sin(phi) * e2)
    return center + length * d


def _emim_template():
    """Approximate 1-ethyl-3-methylimidazolium (C6H11N2+, 19 atoms), centred."""
    rr = 1.36 / (2.0 * math.sin(math.radians(36.0)))
    ang = [math.radians(90.0 + 72.0 * k) for k in range(5)]
    ring = [np.array([rr * math.cos(t), rr * math.sin(t), 0.0]) for t in ang]
    n1, c2, n3, c4, c5 = ring
    atoms = [("N", n1), ("C", c2), ("N", n3), ("C", c4), ("C", c5)]

    def radial(p, length):
        return p + length * p / np.linalg.norm(p)

    atoms += [("H", radial(c2, 1.08)), ("H", radial(c4, 1.08)), ("H", radial(c5, 1.08))]
    c6 = radial(n3, 1.47)                       # methyl on N3
    atoms.append(("C", c6))
    for k in range(3):
        atoms.append(("H", _tetra_arm(n3, c6, 2.0 * math.pi * k / 3.0, 1.09)))
    c7 = radial(n1, 1.47)                       # ethyl CH2 on N1
    atoms.append(("C", c7))
    c8 = _tetra_arm(n1, c7, 0.0, 1.53)
    atoms.append(("C", c8))
    for k in (1, 2):
        atoms.append(("H", _tetra_arm(n1, c7, 2.0 * math.pi * k / 3.0, 1.09)))
    for k in range(3):
        atoms.append(("H", _tetra_arm(c7, c8, math.pi / 3.0 + 2.0 * math.pi * k / 3.0, 1.09)))
    el = [a[0] for a in atoms]
    xyz = np.array([a[1] for a in atoms])
    assert len(el) == 19
    return el, xyz - xyz.mean(axis=0)


def _bf4_template():
    s = 1.40 / math.sqrt(3.0)
    xyz = np.array([[0, 0, 0], [s, s, s], [s, -s, -s], [-s, s, -s], [-s, -s, s]], float)
    return ["B", "F", "F", "F", "F"], xyz


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _min_image_min_dist(new, old, L):
    if len(old) == 0:
        return np.inf
    d = new[:, None, :] - old[None, :, :]
    d -= L * np.round(d / L)
    return float(np.sqrt((d * d).sum(-1)).min())


def emim_pair_mass() -> float:
    el_c, _ = _emim_template()
    el_a, _ = _bf4_template()
    return sum(_MASS[e] for e in el_c + el_a)


def emim_box(n_pairs: int, seed: int, density=1.28, min_sep=0.9, jitter=0.2, tries=4000):
    """EMIM+BF4- box of ``n_pairs`` ion pairs at ``density`` g/cm^3.

    Molecules go to random slots of a g^3 grid (g = ceil((2 n_pairs)^(1/3))) with a
    uniform jitter of +-``jitter`` grid spacings and a uniform random orientation;
    a placement that brings any atom within ``min_sep`` of an already placed atom
    (minimum image) is redrawn.  Returns (pos, species, cell).
    """
    rng = np.random.default_rng([seed, 11])
    L = box_length(n_pairs * emim_pair_mass(), density)
    n_mol = 2 * n_pairs
    g = 1
    while g ** 3 < n_mol:
        g += 1
    h = L / g
    slots = np.array([(i, j, k) for i in range(g) for j in range(g) for k in range(g)], float)
    order = rng.permutation(len(slots))
    kinds = np.array([0] * n_pairs + [1] * n_pairs)
    kinds = kinds[rng.permutation(n_mol)]
    templates = [_emim_template(), _bf4_template()]
    placed_xyz = np.zeros((0, 3))
    placed_el: list[str] = []
    free = list(order)
    for m in range(n_mol):
        el, tpl = templates[kinds[m]]
        ok = False
        for attempt in range(tries):
            slot = free[(attempt // 40) % len(free)]
            centre = (slots[slot] + 0.5 + rng.uniform(-jitter, jitter, 3)) * h
            xyz = tpl @ _random_rotation(rng).T + centre
            xyz = np.mod(xyz, L)
            if _min_image_min_dist(xyz, placed_xyz, L) >= min_sep:
                ok = True
                free.remove(slot)
                break
        if not ok:
            raise RuntimeError(f"emim_box: could not place molecule {m} of {n_mol}")
        placed_xyz = np.concatenate([placed_xyz, xyz])
        placed_el += el
    species = np.array([EMIM_SPECIES[e] for e in placed_el], np.int32)
    return placed_xyz, species, np.eye(3) * L


# --------------------------------------------------------------------------- Li3PO4

LI3PO4_UNIT_MASS = 3 * _MASS["Li"] + _MASS["P"] + 4 * _MASS["O"]


def li3po4_length(n_units: int, density=2.4) -> float:
    return box_length(n_units * LI3PO4_UNIT_MASS, density)


def li3po4_crystal(n_units: int, seed: int, sigma=0.05, density=2.4):
    """Jittered site lattice with Li3PO4 composition (8 atoms per formula unit).

    Sites form an m^3 simple cubic lattice, m the smallest even integer with
    m^3 >= 8 n_units.  Site parity (ix%2, iy%2, iz%2) assigns a 2x2x2 motif:
    (0,0,0) -> P; (1,0,0), (0,1,0), (0,0,1), (1,1,1) -> O; the rest -> Li.  Exactly
    n_units P, 4 n_units O and 3 n_units Li sites are kept (seeded choice), and every
    kept atom is displaced by N(0, sigma^2) per component.
    """
    rng = np.random.default_rng([seed, 21])
    L = li3po4_length(n_units, density)
    m = 2
    while m ** 3 < 8 * n_units:
        m += 2
    idx = np.array([(i, j, k) for i in range(m) for j in range(m) for k in range(m)])
    par = idx % 2
    is_p = (par.sum(1) == 0)
    is_o = ((par.sum(1) == 1) & (par[:, 0] + par[:, 1] + par[:, 2] == 1)) | (par.sum(1) == 3)
    is_li = ~(is_p | is_o)
    keep = []
    spec = []
    for mask, count, s in ((is_li, 3 * n_units, LI3PO4_SPECIES["Li"]),
                           (is_p, n_units, LI3PO4_SPECIES["P"]),
                           (is_o, 4 * n_units, LI3PO4_SPECIES["O"])):
        pool = np.nonzero(mask)[0]
        chosen = np.sort(rng.choice(pool, size=count, replace=False))
        keep.append(chosen)
        spec.append(np.full(count, s, np.int32))
    keep = np.concatenate(keep)
    spec = np.concatenate(spec)
    order = np.argsort(keep, kind="stable")       # spatial (lattice) order
    keep, spec = keep[order], spec[order]
    pos = (idx[keep] + 0.5) * (L / m) + rng.normal(0.0, sigma, (len(keep), 3))
    pos = np.mod(pos, L)
    return pos, spec, np.eye(3) * L


def li3po4_random(n_units: int, seed: int, min_sep=1.5, density=2.4, tries=100000):
    """Random sequential packing of 8 n_units atoms with minimum separation ``min_sep``."""
    rng = np.random.default_rng([seed, 31])
    L = li3po4_length(n_units, density)
    n = 8 * n_units
    pos = np.zeros((n, 3))
    k = 0
    for _ in range(tries * n):
        p = rng.uniform(0.0, L, 3)
        if k:
            d = pos[:k] - p
            d -= L * np.round(d / L)
            if (d * d).sum(1).min() < min_sep * min_sep:
                continue
        pos[k] = p
        k += 1
        if k == n:
            break
    if k < n:
        raise RuntimeError("li3po4_random: packing failed")
    spec = np.array([0] * (3 * n_units) + [1] * n_units + [2] * (4 * n_units), np.int32)
    spec = spec[rng.permutation(n)]
    return pos, spec, np.eye(3) * L


# --------------------------------------------------------------------------- small cases

def dimer(r: float, direction=(0.0, 0.0, 1.0), species=(0, 1), box=100.0):
    """Two atoms at distance r along ``direction`` in a large cubic box."""
    u = np.asarray(direction, float)
    u /= np.linalg.norm(u)
    c = np.full(3, box / 2)
    pos = np.stack([c - 0.5 * r * u, c + 0.5 * r * u])
    return pos, np.asarray(species, np.int32), np.eye(3) * box


def species_masses(kind: str) -> np.ndarray:
    """Atomic masses (amu) indexed by the species numbering of the generators."""
    table = EMIM_SPECIES if kind == "emim" else LI3PO4_SPECIES
    out = np.zeros(len(table))
    for el, idx in table.items():
        out[idx] = _MASS[el]
    return out


def supercell(structure, reps: int):
    """(pos, species, cell) of a reps x reps x reps periodic supercell of one structure."""
    pos, spec, cell = (np.asarray(x) for x in structure)
    shifts = np.array([(i, j, k) for i in range(reps) for j in range(reps) for k in range(reps)], np.float64)
    off = shifts @ cell
    big = (pos[None, :, :] + off[:, None, :]).reshape(-1, 3)
    return big, np.tile(spec, len(shifts)), cell * reps
