"""FP64 CPU oracle of the GMNN energy, forces, virial and parameter gradient.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline / reference leg may import this package.  The GPU library never does, and
this package never imports the GPU library.

``gm_oracle.c`` is the oracle proper (plain loops, FP64, OpenMP over atoms, built with
-ffp-contract=off); ``torch_ref.py`` is an independent restatement in PyTorch FP64 whose
derivatives come from autograd and which cross-checks the hand-derived chain rules.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "gm_oracle.c"
LIB = HERE / "liboracle.so"

_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle into oracle/liboracle.so (gcc, OpenMP, no FP contraction)."""
    if LIB.exists() and not force and LIB.stat().st_mtime >= SRC.stat().st_mtime:
        return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", str(LIB), str(SRC), "-lm"]
    subprocess.run(cmd, check=True)
    return LIB


class _Model(ctypes.Structure):
    _fields_ = [("n_species", ctypes.c_int), ("n_basis", ctypes.c_int), ("n_radial", ctypes.c_int),
                ("n_hidden", ctypes.c_int), ("activation", ctypes.c_int),
                ("r_min", ctypes.c_double), ("r_cut", ctypes.c_double)] + \
               [(k, ctypes.POINTER(ctypes.c_double)) for k in
                ("beta", "W1", "b1", "W2", "b2", "w3", "b3", "sigma", "mu")] + [("basis", ctypes.c_int)]


class _Grad(ctypes.Structure):
    _fields_ = [(k, ctypes.POINTER(ctypes.c_double)) for k in
                ("beta", "W1", "b1", "W2", "b2", "w3", "b3", "sigma", "mu")]


PARAM_NAMES = ("beta", "W1", "b1", "W2", "b2", "w3", "b3", "sigma", "mu")
ACTIVATIONS = {"tanh": 0, "silu": 1}
BASES = {"gaussian": 0, "bessel": 1}


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(str(LIB))
        _lib.or_neighbors.restype = ctypes.c_int
        _lib.or_neighbor_rows.restype = ctypes.c_int
        _lib.or_descriptors.restype = ctypes.c_int
        _lib.or_energy_forces.restype = ctypes.c_int
        _lib.or_param_grad.restype = ctypes.c_int
        _lib.or_loss.restype = ctypes.c_double
        _lib.or_feature_table.restype = ctypes.c_int
        _lib.or_num_threads.restype = ctypes.c_int
        _lib.or_radial_basis.restype = ctypes.c_int
        _lib.or_radial_fns.restype = ctypes.c_int
    return _lib


def _p(a, ct=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


def _model(desc, params, keep):
    arrs = {k: np.ascontiguousarray(params[k], np.float64) for k in PARAM_NAMES}
    keep.extend(arrs.values())
    return _Model(int(desc["n_species"]), int(desc.get("n_basis", 7)), int(desc.get("n_radial", 5)),
                  int(desc["n_hidden"]), ACTIVATIONS[desc.get("activation", "silu")],
                  float(desc.get("r_min", 0.5)), float(desc["r_cut"]),
                  *[_p(arrs[k]) for k in PARAM_NAMES], BASES[desc.get("basis", "gaussian")])


class NeighborList:
    """CSR neighbour list: row_ptr int64 [N+1], col int32 [P], shift int32 [P, 3]."""

    def __init__(self, row_ptr, col, shift):
        self.row_ptr, self.col, self.shift = row_ptr, col, shift

    @property
    def n_pairs(self):
        return int(self.row_ptr[-1])

    def triples(self):
        """Pairs as an int64 [P, 5] array (i, j, n0, n1, n2), sorted lexicographically."""
        n = len(self.row_ptr) - 1
        i = np.repeat(np.arange(n, dtype=np.int64), np.diff(self.row_ptr))
        t = np.column_stack([i, self.col.astype(np.int64), self.shift.astype(np.int64)])
        order = np.lexsort(t.T[::-1])
        return t[order]


def neighbors(batch, r_cut, capacity=None) -> NeighborList:
    """Brute-force O(N^2 x images) neighbour list (FP64, strict r < r_cut)."""
    L = lib()
    pos = np.ascontiguousarray(batch.pos, np.float64)
    cell = np.ascontiguousarray(batch.cell, np.float64).reshape(-1, 9)
    pbc = np.ascontiguousarray(batch.pbc, np.uint8)
    ap = np.ascontiguousarray(batch.atom_ptr, np.int32)
    cap = capacity or max(1024, 200 * batch.n_atoms)
    while True:
        pi = np.empty(cap, np.int32)
        pj = np.empty(cap, np.int32)
        ps = np.empty((cap, 3), np.int32)
        n = ctypes.c_int64(0)
        rc = L.or_neighbors(ctypes.c_int(batch.n_structures), _p(ap, ctypes.c_int), _p(pos), _p(cell),
                            _p(pbc, ctypes.c_ubyte), ctypes.c_double(r_cut), ctypes.c_int64(cap),
                            _p(pi, ctypes.c_int), _p(pj, ctypes.c_int), _p(ps, ctypes.c_int), ctypes.byref(n))
        if rc == 0:
            break
        cap = int(n.value) + 16
    P = int(n.value)
    counts = np.bincount(pi[:P], minlength=batch.n_atoms)
    row_ptr = np.zeros(batch.n_atoms + 1, np.int64)
    row_ptr[1:] = np.cumsum(counts)
    return NeighborList(row_ptr, np.ascontiguousarray(pj[:P]), np.ascontiguousarray(ps[:P]))


def neighbor_rows(batch, r_cut, rows) -> NeighborList:
    """The brute-force neighbour list restricted to the centre atoms in ``rows`` (other
    rows are empty); same rule and arithmetic as neighbors()."""
    L = lib()
    pos = np.ascontiguousarray(batch.pos, np.float64)
    cell = np.ascontiguousarray(batch.cell, np.float64).reshape(-1, 9)
    pbc = np.ascontiguousarray(batch.pbc, np.uint8)
    ap = np.ascontiguousarray(batch.atom_ptr, np.int32)
    rows = np.ascontiguousarray(np.unique(rows), np.int32)
    cap = 400 * len(rows) + 1024
    while True:
        pi = np.empty(cap, np.int32)
        pj = np.empty(cap, np.int32)
        ps = np.empty((cap, 3), np.int32)
        n = ctypes.c_int64(0)
        rc = L.or_neighbor_rows(ctypes.c_int(batch.n_structures), _p(ap, ctypes.c_int), _p(pos), _p(cell),
                                _p(pbc, ctypes.c_ubyte), ctypes.c_double(r_cut), ctypes.c_int(len(rows)),
                                _p(rows, ctypes.c_int), ctypes.c_int64(cap), _p(pi, ctypes.c_int),
                                _p(pj, ctypes.c_int), _p(ps, ctypes.c_int), ctypes.byref(n))
        if rc == 0:
            break
        cap = int(n.value) + 16
    P = int(n.value)
    counts = np.bincount(pi[:P], minlength=batch.n_atoms)
    row_ptr = np.zeros(batch.n_atoms + 1, np.int64)
    row_ptr[1:] = np.cumsum(counts)
    return NeighborList(row_ptr, np.ascontiguousarray(pj[:P]), np.ascontiguousarray(ps[:P]))


def descriptors(batch, desc, params, nl: NeighborList, rows):
    """Moments [len(rows), nr, 20] and features [len(rows), nf] of the atoms in ``rows``."""
    L = lib()
    keep = []
    m = _model(desc, params, keep)
    nr = int(desc.get("n_radial", 5))
    nf = L.or_feature_table(ctypes.c_int(nr), None, None)
    rows = np.ascontiguousarray(rows, np.int32)
    psi = np.zeros((len(rows), nr, 20))
    G = np.zeros((len(rows), nf))
    pos = np.ascontiguousarray(batch.pos, np.float64)
    cell = np.ascontiguousarray(batch.cell, np.float64).reshape(-1, 9)
    spec = np.ascontiguousarray(batch.species, np.int32)
    ap = np.ascontiguousarray(batch.atom_ptr, np.int32)
    rp = np.ascontiguousarray(nl.row_ptr, np.int64)
    col = np.ascontiguousarray(nl.col, np.int32)
    sh = np.ascontiguousarray(nl.shift, np.int32)
    rc = L.or_descriptors(ctypes.byref(m), ctypes.c_int(batch.n_structures), _p(ap, ctypes.c_int), _p(pos),
                          _p(spec, ctypes.c_int), _p(cell), _p(rp, ctypes.c_int64), _p(col, ctypes.c_int),
                          _p(sh, ctypes.c_int), ctypes.c_int(len(rows)), _p(rows, ctypes.c_int), _p(psi), _p(G))
    if rc != 0:
        raise RuntimeError(f"or_descriptors failed ({rc})")
    return psi, G


def energy_forces(batch, desc, params, nl: NeighborList, virial=True, psi=False, features=False):
    """Energies (per structure and per atom), forces, virials and optional intermediates."""
    L = lib()
    keep = []
    m = _model(desc, params, keep)
    N, B = batch.n_atoms, batch.n_structures
    nr = int(desc.get("n_radial", 5))
    nf = L.or_feature_table(ctypes.c_int(nr), None, None)
    out = {"E": np.zeros(B), "E_atom": np.zeros(N), "F": np.zeros((N, 3))}
    out["virial"] = np.zeros((B, 3, 3)) if virial else None
    out["psi"] = np.zeros((N, nr, 20)) if psi else None
    out["G"] = np.zeros((N, nf)) if features else None
    pos = np.ascontiguousarray(batch.pos, np.float64)
    cell = np.ascontiguousarray(batch.cell, np.float64).reshape(-1, 9)
    spec = np.ascontiguousarray(batch.species, np.int32)
    ap = np.ascontiguousarray(batch.atom_ptr, np.int32)
    rp = np.ascontiguousarray(nl.row_ptr, np.int64)
    col = np.ascontiguousarray(nl.col, np.int32)
    sh = np.ascontiguousarray(nl.shift, np.int32)
    rc = L.or_energy_forces(ctypes.byref(m), ctypes.c_int(B), _p(ap, ctypes.c_int), _p(pos),
                            _p(spec, ctypes.c_int), _p(cell), _p(rp, ctypes.c_int64), _p(col, ctypes.c_int),
                            _p(sh, ctypes.c_int), _p(out["E"]), _p(out["E_atom"]), _p(out["F"]),
                            _p(out["virial"]), _p(out["psi"]), _p(out["G"]))
    if rc != 0:
        raise RuntimeError(f"or_energy_forces failed ({rc})")
    return out


def energy_forces_ensemble(batch, desc, params, nl: NeighborList, virial=True):
    """Shallow ensemble (section "Uncertainty Quantification"): output weights w3 [H, E] and
    b3 [E] on one network.  Head k is the model with w3[:, k] and b3[k]; each head is evaluated
    in full (energies, forces, virials), then the mean over heads gives the ensemble energy
    and force (Eq. jacobian: the mean force is minus the gradient of the mean energy) and the
    spread over heads with the 1/E normalisation of Eq. uncertainty: per structure for the
    energy, per atom for the force with the sum over its three components.
    Returns E [B], F [N,3], virial [B,3,3], E_heads [B,E], F_heads [E,N,3], E_std [B], F_std [N]."""
    w3 = np.asarray(params["w3"], np.float64)
    b3 = np.asarray(params["b3"], np.float64).reshape(-1)
    if w3.ndim == 1:
        w3 = w3[:, None]
    n_heads = w3.shape[1]
    heads = [energy_forces(batch, desc, dict(params, w3=np.ascontiguousarray(w3[:, k]), b3=b3[k:k + 1]), nl,
                           virial=virial) for k in range(n_heads)]
    Eh = np.stack([h["E"] for h in heads], 1)
    Fh = np.stack([h["F"] for h in heads])
    Em, Fm = Eh.mean(1), Fh.mean(0)
    out = {"E_heads": Eh, "F_heads": Fh, "E": Em, "F": Fm,
           "E_std": np.sqrt(((Eh - Em[:, None]) ** 2).mean(1)),
           "F_std": np.sqrt(((Fh - Fm[None]) ** 2).sum(2).mean(0)),
           "E_atom": np.mean([h["E_atom"] for h in heads], 0)}
    out["virial"] = np.mean([h["virial"] for h in heads], 0) if virial else None
    return out


class _SubBatch:
    """The attributes of a batch the oracle reads (positions, species, cells, atom ranges)."""

    def __init__(self, pos, species, atom_ptr, cell, pbc):
        self.pos, self.species, self.atom_ptr, self.cell, self.pbc = pos, species, atom_ptr, cell, pbc
        self.n_atoms = int(atom_ptr[-1])
        self.n_structures = int(len(atom_ptr) - 1)


def sampled_forces(batch, desc, params, rows):
    """Exact forces F[rows] and atomic energies E_atom[rows] of a few atoms of a large system.

    F_i = -d/dr_i sum_k E_k involves only the atoms k whose environment holds i, i.e. i itself
    and its neighbours (the neighbour relation is symmetric), and E_k needs k's full neighbour
    row.  So the model is evaluated on the sub-system of those atoms K and their neighbours,
    with complete rows for K and empty rows for the rest (same positions and cells, so the
    image shifts stay valid).  Nothing is approximated: F[rows] and E_atom[rows] equal the
    full evaluation's up to summation order."""
    r_cut = float(desc["r_cut"])
    rows = np.unique(np.asarray(rows, np.int64))
    first = neighbor_rows(batch, r_cut, rows)
    K = np.unique(np.concatenate([rows, first.col.astype(np.int64)]))
    nlK = neighbor_rows(batch, r_cut, K)
    U = np.unique(np.concatenate([K, nlK.col.astype(np.int64)]))
    remap = np.full(batch.n_atoms, -1, np.int64)
    remap[U] = np.arange(len(U))
    counts = np.diff(nlK.row_ptr)[U]
    row_ptr = np.zeros(len(U) + 1, np.int64)
    row_ptr[1:] = np.cumsum(counts)
    # nlK's rows are contiguous in global atom order and U is ascending, so the pairs keep
    # their order; only the column indices are renumbered
    col = remap[nlK.col.astype(np.int64)].astype(np.int32)
    ap = np.asarray(batch.atom_ptr, np.int64)
    sub_ap = np.searchsorted(U, ap).astype(np.int32)
    sub = _SubBatch(np.ascontiguousarray(np.asarray(batch.pos)[U]), np.ascontiguousarray(np.asarray(batch.species)[U]),
                    sub_ap, np.asarray(batch.cell), np.asarray(batch.pbc))
    out = energy_forces(sub, desc, params, NeighborList(row_ptr, col, nlK.shift), virial=False)
    return {"rows": rows, "F": out["F"][remap[rows]], "E_atom": out["E_atom"][remap[rows]],
            "n_sub_atoms": len(U), "n_complete_rows": len(K)}


def loss(batch, E, E_ref, F, F_ref, wE=1.0, wF=1.0):
    """Force-matching loss and its gradients (gE [B], gF [N, 3])."""
    L = lib()
    ap = np.ascontiguousarray(batch.atom_ptr, np.int32)
    gE = np.zeros(batch.n_structures)
    gF = np.zeros((batch.n_atoms, 3))
    arrs = [np.ascontiguousarray(a, np.float64) for a in (E, E_ref, F, F_ref)]
    val = L.or_loss(ctypes.c_int(batch.n_structures), _p(ap, ctypes.c_int), *[_p(a) for a in arrs],
                    ctypes.c_double(wE), ctypes.c_double(wF), _p(gE), _p(gF))
    return val, gE, gF


def param_grad(batch, desc, params, nl: NeighborList, gE, gF):
    """d/dtheta of sum_b gE_b E_b + sum_i gF_i . F_i, as a dict of named arrays."""
    L = lib()
    keep = []
    m = _model(desc, params, keep)
    grads = {k: np.zeros_like(np.asarray(params[k], np.float64)) for k in PARAM_NAMES}
    g = _Grad(*[_p(grads[k]) for k in PARAM_NAMES])
    pos = np.ascontiguousarray(batch.pos, np.float64)
    cell = np.ascontiguousarray(batch.cell, np.float64).reshape(-1, 9)
    spec = np.ascontiguousarray(batch.species, np.int32)
    ap = np.ascontiguousarray(batch.atom_ptr, np.int32)
    rp = np.ascontiguousarray(nl.row_ptr, np.int64)
    col = np.ascontiguousarray(nl.col, np.int32)
    sh = np.ascontiguousarray(nl.shift, np.int32)
    gE = np.ascontiguousarray(gE, np.float64)
    gF = np.ascontiguousarray(gF, np.float64).reshape(-1, 3)
    rc = L.or_param_grad(ctypes.byref(m), ctypes.c_int(batch.n_structures), _p(ap, ctypes.c_int), _p(pos),
                         _p(spec, ctypes.c_int), _p(cell), _p(rp, ctypes.c_int64), _p(col, ctypes.c_int),
                         _p(sh, ctypes.c_int), _p(gE), _p(gF), ctypes.byref(g))
    if rc != 0:
        raise RuntimeError(f"or_param_grad failed ({rc})")
    return grads


def radial_basis(desc, params, r):
    """(B, dB): f_c(r) Phi_k(r) and its r-derivative for k < n_basis, at one distance."""
    L = lib()
    keep = []
    m = _model(desc, params, keep)
    nb = int(desc.get("n_basis", 7))
    B, dB = np.zeros(nb), np.zeros(nb)
    rc = L.or_radial_basis(ctypes.byref(m), ctypes.c_double(r), _p(B), _p(dB))
    if rc != 0:
        raise RuntimeError(f"or_radial_basis failed ({rc})")
    return B, dB


def radial_fns(desc, params, zi, zj, r):
    """(R, dR): the radial functions R_s(r) of the ordered species pair (zi, zj) and dR_s/dr."""
    L = lib()
    keep = []
    m = _model(desc, params, keep)
    nr = int(desc.get("n_radial", 5))
    R, dR = np.zeros(nr), np.zeros(nr)
    rc = L.or_radial_fns(ctypes.byref(m), ctypes.c_int(zi), ctypes.c_int(zj), ctypes.c_double(r), _p(R), _p(dR))
    if rc != 0:
        raise RuntimeError(f"or_radial_fns failed ({rc})")
    return R, dR


def feature_table(n_radial=5):
    """(family [F], tensor-state offsets [F, 3]) of the contraction features."""
    L = lib()
    nf = L.or_feature_table(ctypes.c_int(n_radial), None, None)
    fam = np.zeros(nf, np.int32)
    off = np.zeros((nf, 3), np.int32)
    L.or_feature_table(ctypes.c_int(n_radial), _p(fam, ctypes.c_int), _p(off, ctypes.c_int))
    return fam, off


def num_threads():
    return int(lib().or_num_threads())


def set_threads(n: int):
    """OpenMP threads of the oracle's later calls in this process."""
    lib().or_set_threads(ctypes.c_int(int(n)))


def omp_env(threads: int | None):
    """Environment for a child process that should use ``threads`` OpenMP threads."""
    env = dict(os.environ)
    if threads:
        env["OMP_NUM_THREADS"] = str(threads)
    return env
