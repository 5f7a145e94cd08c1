"""CPU pins of the FP64 oracle against what the paper and the mathematics fix.

Each test pins the oracle to something other than itself: finite differences (forces,
virial, parameter gradient), invariances and extensivity (stated for the descriptor and
the additive energy in the paper's Methods), closed forms of special configurations,
identities that hold for any configuration, brute force and textbook lattice counts, and
an independent autograd restatement (oracle/torch_ref.py).
"""
from pathlib import Path

import numpy as np
import pytest

import oracle
import synth
from oracle import torch_ref
from synth.systems import make_batch, dimer

GOLDEN = Path(__file__).resolve().parent / "golden"


@pytest.fixture(scope="module")
def cfg1():
    b, d, p = synth.config(1, activation="tanh")
    return b, d, p


def _single(pos, spec, cell, n_species):
    return make_batch([(pos, spec, cell)], n_species)


def _ef(batch, desc, params, **kw):
    nl = oracle.neighbors(batch, desc["r_cut"])
    return oracle.energy_forces(batch, desc, params, nl, **kw), nl


# ----------------------------------------------------------------- neighbour rule

def _sc_counts():
    rows = [l.split() for l in (GOLDEN / "sc_coordination.txt").read_text().splitlines()
            if l.strip() and not l.startswith("#")]
    return [(float(a), int(b)) for a, b in rows]


@pytest.mark.parametrize("rc,count", _sc_counts())
def test_sc_lattice_self_images(rc, count):
    """One atom in a unit cube: its neighbours are its own periodic images."""
    b = _single(np.array([[0.3, 0.6, 0.9]]), np.array([0]), np.eye(3), 1)
    nl = oracle.neighbors(b, rc)
    assert nl.n_pairs == count


@pytest.mark.parametrize("rc,count", _sc_counts()[:4])
def test_sc_lattice_supercell_and_triclinic_basis(rc, count):
    """2x2x2 supercell and a sheared basis of the same lattice give the same counts."""
    g = np.array([(i, j, k) for i in range(2) for j in range(2) for k in range(2)], float)
    b = _single(g + 0.25, np.zeros(8, int), 2 * np.eye(3), 1)
    nl = oracle.neighbors(b, rc)
    assert np.all(np.diff(nl.row_ptr) == count)
    sheared = np.array([[1.0, 0, 0], [1.0, 1.0, 0], [0, 0, 1.0]])
    b2 = _single(np.array([[0.1, 0.2, 0.3]]), np.array([0]), sheared, 1)
    assert oracle.neighbors(b2, rc).n_pairs == count


def test_cutoff_is_strict():
    """A pair at exactly r_cut is excluded (f_c(r_cut) = 0, so E is unaffected)."""
    b = _single(np.array([[0.0, 0.0, 0.0], [2.5, 0.0, 0.0]]), np.array([0, 0]), 20 * np.eye(3), 1)
    assert oracle.neighbors(b, 2.5).n_pairs == 0
    assert oracle.neighbors(b, np.nextafter(2.5, 3.0)).n_pairs == 2


def test_neighbors_brute_force_numpy_and_symmetry():
    """Random small boxes (some below 2 r_cut): set equals an independent numpy brute force
    over a wide image range; (i, j, n) present iff (j, i, -n) present."""
    rng = np.random.default_rng(7)
    for L, n, rc in ((4.0, 5, 3.0), (7.0, 20, 3.5), (2.5, 3, 3.1)):
        pos = rng.uniform(-L, 2 * L, (n, 3))          # deliberately outside the cell
        b = _single(pos, np.zeros(n, int), L * np.eye(3), 1)
        nl = oracle.neighbors(b, rc)
        got = {tuple(t) for t in nl.triples()}
        want = set()
        K = int(np.ceil(rc / L)) + 3
        for i in range(n):
            for j in range(n):
                for s in np.ndindex(2 * K + 1, 2 * K + 1, 2 * K + 1):
                    sh = np.array(s) - K - np.floor(pos[j] / L).astype(int) + np.floor(pos[i] / L).astype(int)
                    d = pos[j] - pos[i] + sh * L
                    if (i != j or np.any(sh != 0)) and d @ d < rc * rc:
                        want.add((i, j, *map(int, sh)))
        assert got == want
        assert {(j, i, -a, -b_, -c) for (i, j, a, b_, c) in got} == got


# ----------------------------------------------------------------- forces / virial

def _fd_forces(batch, desc, params, atoms, h=1e-5):
    out = np.zeros((len(atoms), 3))
    for q, k in enumerate(atoms):
        for c in range(3):
            e = []
            for sgn in (1, -1):
                b2 = make_batch([(batch.pos.copy(), batch.species, batch.cell[0])], batch.n_species)
                b2.pos[k, c] += sgn * h
                e.append(_ef(b2, desc, params, virial=False)[0]["E"][0])
            out[q, c] = -(e[0] - e[1]) / (2 * h)
    return out


@pytest.mark.parametrize("act", ["tanh", "silu"])
def test_forces_match_central_differences(cfg1, act):
    b, d, p = cfg1
    d = dict(d, activation=act)
    out, _ = _ef(b, d, p)
    atoms = [0, 17, 50, 95]
    fd = _fd_forces(b, d, p, atoms)
    frms = np.sqrt((out["F"] ** 2).mean())
    err = np.abs(fd - out["F"][atoms])
    assert err.max() <= 1e-6 * max(frms, np.abs(out["F"][atoms]).max())


FAMILY_SLICES = [(0, 5), (5, 20), (20, 35), (35, 50), (50, 85), (85, 160), (160, 235), (235, 360)]


@pytest.mark.parametrize("fam", range(8))
def test_forces_per_contraction_family(cfg1, fam):
    """E built from one contraction family at a time: each family's backward is pinned
    separately by finite differences."""
    b, d, p = cfg1
    lo, hi = FAMILY_SLICES[fam]
    p2 = dict(p)
    W1 = np.zeros_like(p["W1"])
    W1[lo:hi] = p["W1"][lo:hi] * 30.0
    p2["W1"] = W1
    out, _ = _ef(b, d, p2)
    atoms = [3, 60]
    fd = _fd_forces(b, d, p2, atoms)
    assert np.abs(out["F"][atoms]).max() > 1e-6
    assert np.abs(fd - out["F"][atoms]).max() <= 1e-6 * np.abs(out["F"][atoms]).max() + 1e-12


def test_zero_net_force_and_symmetric_virial(cfg1):
    b, d, p = cfg1
    out, _ = _ef(b, d, p)
    frms = np.sqrt((out["F"] ** 2).mean())
    assert np.abs(out["F"].sum(0)).max() <= 1e-10 * b.n_atoms * frms
    W = out["virial"][0]
    assert np.abs(W - W.T).max() <= 1e-12 * np.abs(W).max()


def test_virial_matches_strain_differences(cfg1):
    """virial = -dE/d(strain) with x -> x (I + eps) applied to positions and cell."""
    b, d, p = cfg1
    out, _ = _ef(b, d, p)
    h = 1e-6
    for (a, c) in ((0, 0), (1, 2), (2, 1), (2, 2)):
        e = []
        for sgn in (1, -1):
            eps = np.zeros((3, 3))
            eps[a, c] = sgn * h
            D = np.eye(3) + eps
            b2 = make_batch([(b.pos @ D, b.species, b.cell[0] @ D)], b.n_species)
            e.append(_ef(b2, d, p, virial=False)[0]["E"][0])
        fd = -(e[0] - e[1]) / (2 * h)
        assert abs(fd - out["virial"][0][a, c]) <= 1e-6 * np.abs(out["virial"]).max()


# ----------------------------------------------------------------- invariances

def _rotation(seed):
    rng = np.random.default_rng(seed)
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def test_rotation_invariance_periodic(cfg1):
    """Rotating positions and lattice vectors together (a triclinic cell in the lab
    frame) leaves E unchanged and rotates F."""
    b, d, p = cfg1
    ref, _ = _ef(b, d, p)
    for seed in (1, 2):
        Q = _rotation(seed)
        b2 = make_batch([(b.pos @ Q.T, b.species, b.cell[0] @ Q.T)], b.n_species)
        out, _ = _ef(b2, d, p)
        assert abs(out["E"][0] - ref["E"][0]) <= 1e-12 * np.abs(ref["E_atom"]).sum()
        assert np.abs(out["F"] - ref["F"] @ Q.T).max() <= 1e-10 * np.abs(ref["F"]).max()
    # improper rotation (reflection): the invariants are O(3) invariants
    Pm = np.diag([1.0, -1.0, 1.0]) @ _rotation(3)
    b3 = make_batch([(b.pos @ Pm.T, b.species, b.cell[0] @ Pm.T)], b.n_species)
    out, _ = _ef(b3, d, p)
    assert abs(out["E"][0] - ref["E"][0]) <= 1e-12 * np.abs(ref["E_atom"]).sum()


def test_translation_permutation_and_lattice_shift(cfg1):
    b, d, p = cfg1
    ref, _ = _ef(b, d, p)
    tol = 1e-12 * np.abs(ref["E_atom"]).sum()
    bt = make_batch([(b.pos + np.array([3.3, -7.1, 0.4]), b.species, b.cell[0])], b.n_species)
    out, _ = _ef(bt, d, p)
    assert abs(out["E"][0] - ref["E"][0]) <= tol
    perm = np.random.default_rng(3).permutation(b.n_atoms)
    bp = make_batch([(b.pos[perm], b.species[perm], b.cell[0])], b.n_species)
    out, _ = _ef(bp, d, p)
    assert abs(out["E"][0] - ref["E"][0]) <= tol
    assert np.abs(out["F"] - ref["F"][perm]).max() <= 1e-12 * np.abs(ref["F"]).max() * 10
    pos = b.pos.copy()
    pos[5] += b.cell[0][0] * 2 - b.cell[0][2]
    bs = make_batch([(pos, b.species, b.cell[0])], b.n_species)
    out, _ = _ef(bs, d, p)
    assert abs(out["E"][0] - ref["E"][0]) <= tol
    assert np.abs(out["F"] - ref["F"]).max() <= 1e-10 * np.abs(ref["F"]).max()


def test_extensivity(cfg1):
    """Periodic 2x1x1 replica gives 2E; two copies of a molecule farther apart than r_cut
    give twice the energy of one."""
    b, d, p = cfg1
    ref, _ = _ef(b, d, p)
    L = b.cell[0]
    pos2 = np.concatenate([b.pos, b.pos + L[0]])
    cell2 = L.copy()
    cell2[0] *= 2
    b2 = make_batch([(pos2, np.concatenate([b.species, b.species]), cell2)], b.n_species)
    out, _ = _ef(b2, d, p)
    assert abs(out["E"][0] - 2 * ref["E"][0]) <= 1e-12 * 2 * np.abs(ref["E_atom"]).sum()
    assert np.abs(out["F"][: b.n_atoms] - ref["F"]).max() <= 1e-10 * np.abs(ref["F"]).max()
    # isolated molecule: the first 19 atoms of a fresh template box
    from synth.systems import _emim_template
    el, xyz = _emim_template()
    spec = np.array([synth.EMIM_SPECIES[e] for e in el])
    big = 60.0 * np.eye(3)
    one = _ef(_single(xyz + 10.0, spec, big, 5), d, p)[0]["E"][0]
    two = _ef(_single(np.concatenate([xyz + 10.0, xyz + 10.0 + np.array([d["r_cut"] + 8.0, 0, 0])]),
                      np.concatenate([spec, spec]), big, 5), d, p)[0]["E"][0]
    assert abs(two - 2 * one) <= 1e-12 * abs(one) * 10


# ----------------------------------------------------------------- closed forms

def _mlp_np(x, p, act):
    f = np.tanh if act == "tanh" else (lambda z: z / (1.0 + np.exp(-z)))
    return f(f(x @ p["W1"] + p["b1"]) @ p["W2"] + p["b2"]) @ p["w3"] + p["b3"][0]


@pytest.mark.parametrize("act", ["tanh", "silu"])
def test_isolated_atom_energy(cfg1, act):
    """No neighbour: G = 0 and E = sigma_Z NN(0) + mu_Z (Eq. scale_shift)."""
    _, d, p = cfg1
    d = dict(d, activation=act)
    for z in range(5):
        out, nl = _ef(_single(np.array([[1.0, 2.0, 3.0]]), np.array([z]), 30 * np.eye(3), 5), d, p)
        assert nl.n_pairs == 0
        want = p["sigma"][z] * _mlp_np(np.zeros(360), p, act) + p["mu"][z]
        assert abs(out["E"][0] - want) <= 1e-13 * max(1.0, abs(want))
        assert np.all(out["F"] == 0.0)


def test_dimer_moments_and_features(cfg1):
    """Dimer: Psi_L = R u^(x)L, so every feature is a product of rank-0 moments."""
    _, d, p = cfg1
    u = np.array([0.3, -0.5, 0.81])
    u /= np.linalg.norm(u)
    pos, spec, cell = dimer(2.7, u, (1, 2))
    out, _ = _ef(_single(pos, spec, cell, 5), d, p, psi=True, features=True)
    psi = out["psi"][0]
    R = psi[:, 0]
    assert np.all(np.abs(R) > 1e-3)
    ux, uy, uz = u
    m1 = np.array([ux, uy, uz])
    m2 = np.array([ux * ux, ux * uy, ux * uz, uy * uy, uy * uz, uz * uz])
    m3 = np.array([ux ** 3, ux * ux * uy, ux * ux * uz, ux * uy * uy, ux * uy * uz, ux * uz * uz,
                   uy ** 3, uy * uy * uz, uy * uz * uz, uz ** 3])
    assert np.allclose(psi[:, 1:4], R[:, None] * m1, rtol=0, atol=1e-14)
    assert np.allclose(psi[:, 4:10], R[:, None] * m2, rtol=0, atol=1e-14)
    assert np.allclose(psi[:, 10:20], R[:, None] * m3, rtol=0, atol=1e-14)
    G = out["G"][0]
    want = [R[s] for s in range(5)]
    for _ in range(3):
        want += [R[a] * R[b_] for a in range(5) for b_ in range(a, 5)]
    want += [R[a] * R[b_] * R[c] for a in range(5) for b_ in range(a, 5) for c in range(b_, 5)]
    want += [R[a] * R[b_] * R[c] for a in range(5) for b_ in range(5) for c in range(a, 5)]
    want += [R[a] * R[b_] * R[c] for a in range(5) for b_ in range(a, 5) for c in range(5)]
    want += [R[a] * R[b_] * R[c] for a in range(5) for b_ in range(5) for c in range(5)]
    assert np.allclose(G, want, rtol=1e-13, atol=1e-16)


def _centre_features(r_a, r_b, u_a, u_b, d, p, spec=(0, 1, 3)):
    pos = np.array([[20.0, 20.0, 20.0], [20.0, 20.0, 20.0] + r_a * np.asarray(u_a),
                    [20.0, 20.0, 20.0] + r_b * np.asarray(u_b)])
    out, _ = _ef(_single(pos, np.array(spec), 40 * np.eye(3), 5), d, p, features=True, psi=True)
    return out["G"][0], out["psi"][0]


def test_axis_configurations_pin_slots_and_topology(cfg1):
    """Centre with two neighbours along +x/-x (pins which slot carries which rank) and
    along +x/+y (pins the index topology of each family), against closed forms in the
    rank-0 moments a, b of the two dimers."""
    _, d, p = cfg1
    ra, rb = 1.9, 3.1
    a = _centre_features(ra, 30.0, [1, 0, 0], [0, 1, 0], d, p)[1][:, 0]   # only A in range
    b_ = _centre_features(30.0, rb, [1, 0, 0], [0, 1, 0], d, p)[1][:, 0]  # only B in range
    r5 = range(5)

    def feats(X, Y, Z):
        """Family-ordered products given per-family rank factors."""
        out = [X[0][s] for s in r5]
        for fam in (1, 2, 3):
            out += [X[fam](s, t) for s in r5 for t in range(s, 5)]
        out += [Y[0](s, t, v) for s in r5 for t in range(s, 5) for v in range(t, 5)]
        out += [Y[1](s, t, v) for s in r5 for t in r5 for v in range(s, 5)]
        out += [Y[2](s, t, v) for s in r5 for t in range(s, 5) for v in r5]
        out += [Y[3](s, t, v) for s in r5 for t in r5 for v in r5]
        return np.array(out)

    # +x / -x
    G, _ = _centre_features(ra, rb, [1, 0, 0], [-1, 0, 0], d, p)
    P, Mm = a + b_, a - b_
    want = feats([P, lambda s, t: Mm[s] * Mm[t], lambda s, t: P[s] * P[t], lambda s, t: Mm[s] * Mm[t]],
                 [lambda s, t, v: P[s] * P[t] * P[v], lambda s, t, v: Mm[s] * P[t] * Mm[v],
                  lambda s, t, v: Mm[s] * Mm[t] * P[v], lambda s, t, v: Mm[s] * Mm[t] * P[v]], None)
    assert np.allclose(G, want, rtol=1e-12, atol=1e-15)
    # +x / +y
    G, _ = _centre_features(ra, rb, [1, 0, 0], [0, 1, 0], d, p)
    two = lambda s, t: a[s] * a[t] + b_[s] * b_[t]
    three = lambda s, t, v: a[s] * a[t] * a[v] + b_[s] * b_[t] * b_[v]
    want = feats([a + b_, two, two, two], [three, three, three, three], None)
    assert np.allclose(G, want, rtol=1e-12, atol=1e-15)


def test_trace_identities_any_configuration(cfg1):
    """sum_a (Psi2)_aa = Psi0 and sum_a (Psi3)_aac = (Psi1)_c, since |rhat| = 1."""
    b, d, p = cfg1
    out, _ = _ef(b, d, p, psi=True)
    psi = out["psi"]
    tr2 = psi[..., 4] + psi[..., 7] + psi[..., 9]
    assert np.allclose(tr2, psi[..., 0], rtol=0, atol=1e-13)
    t3 = np.stack([psi[..., 10] + psi[..., 13] + psi[..., 15],
                   psi[..., 11] + psi[..., 16] + psi[..., 18],
                   psi[..., 12] + psi[..., 17] + psi[..., 19]], -1)
    assert np.allclose(t3, psi[..., 1:4], rtol=0, atol=1e-13)


def test_synthetic_parameters_keep_activations_unsaturated(cfg1):
    b, d, p = cfg1
    out, _ = _ef(b, d, p, features=True)
    z = out["G"] @ p["W1"] + p["b1"]
    assert (np.abs(z) < 3).mean() >= 0.5
    rms = [np.sqrt((out["G"][:, lo:hi] ** 2).mean()) for lo, hi in FAMILY_SLICES]
    assert min(rms) > 1e-2          # every contraction family contributes


# ----------------------------------------------------------------- autograd + gradient

@pytest.mark.parametrize("act", ["tanh", "silu"])
def test_oracle_matches_autograd_restatement(cfg1, act):
    b, d, p = cfg1
    d = dict(d, activation=act)
    out, nl = _ef(b, d, p, features=True)
    t = torch_ref.energy_forces(b, d, p, nl)
    assert abs(out["E"][0] - t["E"][0]) <= 1e-12 * np.abs(t["E_atom"]).sum()
    assert np.abs(out["F"] - t["F"]).max() <= 1e-12 * np.abs(t["F"]).max()
    assert np.abs(out["virial"] - t["virial"]).max() <= 1e-12 * np.abs(t["virial"]).max()
    assert np.abs(out["G"] - t["G"]).max() <= 1e-13


def _loss_setup(b, d, p, nl):
    out = oracle.energy_forces(b, d, p, nl)
    rng = np.random.default_rng(11)
    Eref = out["E"] + rng.normal(0, 0.5, out["E"].shape)
    Fref = out["F"] + rng.normal(0, 0.1, out["F"].shape)
    return Eref, Fref


def _loss_value(b, d, p, nl, Eref, Fref):
    out = oracle.energy_forces(b, d, p, nl, virial=False)
    return oracle.loss(b, out["E"], Eref, out["F"], Fref)


@pytest.mark.parametrize("act", ["tanh", "silu"])
def test_param_grad_matches_autograd(cfg1, act):
    b, d, p = cfg1
    d = dict(d, activation=act)
    nl = oracle.neighbors(b, d["r_cut"])
    Eref, Fref = _loss_setup(b, d, p, nl)
    _, gE, gF = _loss_value(b, d, p, nl, Eref, Fref)
    g = oracle.param_grad(b, d, p, nl, gE, gF)
    _, gt = torch_ref.loss_param_grad(b, d, p, nl, Eref, Fref)
    for k in g:
        assert np.abs(g[k] - gt[k]).max() <= 1e-11 * np.abs(gt[k]).max() + 1e-300, k


def test_param_grad_matches_finite_differences(cfg1):
    b, d, p = cfg1
    nl = oracle.neighbors(b, d["r_cut"])
    Eref, Fref = _loss_setup(b, d, p, nl)
    _, gE, gF = _loss_value(b, d, p, nl, Eref, Fref)
    g = oracle.param_grad(b, d, p, nl, gE, gF)
    rng = np.random.default_rng(5)
    for k in g:
        flat = g[k].reshape(-1)
        cand = np.argsort(-np.abs(flat))[:2].tolist() + rng.integers(0, flat.size, 1).tolist()
        for e in cand:
            h = 1e-6 * max(1.0, abs(p[k].reshape(-1)[e]))
            vals = []
            for sgn in (1, -1):
                p2 = {q: v.copy() for q, v in p.items()}
                p2[k].reshape(-1)[e] += sgn * h
                vals.append(_loss_value(b, d, p2, nl, Eref, Fref)[0])
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - flat[e]) <= 1e-5 * np.abs(flat).max() + 1e-12, (k, e, fd, flat[e])


def test_row_subset_functions_agree_with_full_oracle(cfg1):
    """The sampled-row neighbour list and descriptors used for full-size checks are the
    rows of the full oracle, bit for bit."""
    b, d, p = cfg1
    nl = oracle.neighbors(b, d["r_cut"])
    rows = [0, 13, 50, 95]
    part = oracle.neighbor_rows(b, d["r_cut"], rows)
    full = nl.triples()
    assert np.array_equal(full[np.isin(full[:, 0], rows)], part.triples())
    psi, G = oracle.descriptors(b, d, p, part, rows)
    ref = oracle.energy_forces(b, d, p, nl, psi=True, features=True)
    assert np.array_equal(psi, ref["psi"][rows]) and np.array_equal(G, ref["G"][rows])
