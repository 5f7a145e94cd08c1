"""CPU pins of the oracle's shallow-ensemble readout (section "Uncertainty Quantification").

E heads share the network up to the last hidden layer; the ensemble energy is the mean of
the heads' energies and the ensemble force is the gradient of that mean, which equals the
mean of the heads' forces (Eq. jacobian); the uncertainty is the spread over heads with the
1/E normalisation (Eq. uncertainty).  Pinned by: one head reproducing the plain model,
central differences of the mean energy, the closed form of the spread of two heads
(|x1 - x2| / 2), heads that agree having no spread, and invariance under reordering heads.
"""
import numpy as np
import pytest

import oracle
import synth
from synth.params import make_params
from synth.systems import make_batch


@pytest.fixture(scope="module")
def setup():
    b, d, p = synth.config(1, activation="tanh")
    nl = oracle.neighbors(b, d["r_cut"])
    pe = make_params(d["n_species"], d["n_hidden"], 1001, 40.0, n_ensemble=3)
    pe["beta"] = p["beta"]
    return b, d, p, pe, nl


def test_single_head_is_the_plain_model(setup):
    b, d, p, _, nl = setup
    one = dict(p, w3=np.asarray(p["w3"])[:, None], b3=np.asarray(p["b3"]))
    e = oracle.energy_forces_ensemble(b, d, one, nl)
    ref = oracle.energy_forces(b, d, p, nl)
    assert np.array_equal(e["E"], ref["E"]) and np.array_equal(e["F"], ref["F"])
    assert np.all(e["E_std"] == 0.0) and np.all(e["F_std"] == 0.0)


def test_mean_force_is_minus_the_gradient_of_the_mean_energy(setup):
    b, d, _, pe, nl = setup
    out = oracle.energy_forces_ensemble(b, d, pe, nl, virial=False)
    h = 1e-5
    for k in (2, 47, 90):
        for c in range(3):
            e = []
            for sgn in (1, -1):
                pos = b.pos.copy()
                pos[k, c] += sgn * h
                b2 = make_batch([(pos, b.species, b.cell[0])], b.n_species)
                e.append(oracle.energy_forces_ensemble(b2, d, pe, nl, virial=False)["E"][0])
            fd = -(e[0] - e[1]) / (2 * h)
            assert abs(fd - out["F"][k, c]) <= 1e-6 * np.abs(out["F"]).max(), (k, c)


def test_two_heads_spread_closed_form(setup):
    """For two heads the 1/E spread is half their difference: sigma = |x1 - x2| / 2."""
    b, d, _, pe, nl = setup
    two = dict(pe, w3=np.asarray(pe["w3"])[:, :2].copy(), b3=np.asarray(pe["b3"])[:2].copy())
    out = oracle.energy_forces_ensemble(b, d, two, nl, virial=False)
    assert np.allclose(out["E_std"], np.abs(out["E_heads"][:, 0] - out["E_heads"][:, 1]) / 2, rtol=1e-12)
    dF = np.linalg.norm(out["F_heads"][0] - out["F_heads"][1], axis=1)
    assert np.allclose(out["F_std"], dF / 2, rtol=1e-10, atol=1e-14)
    assert out["E_std"].min() > 0 and out["F_std"].max() > 0


def test_agreeing_heads_have_no_spread_and_order_does_not_matter(setup):
    b, d, p, pe, nl = setup
    w = np.asarray(p["w3"])
    same = dict(p, w3=np.stack([w, w, w], 1), b3=np.full(3, np.asarray(p["b3"])[0]))
    out = oracle.energy_forces_ensemble(b, d, same, nl)
    ref = oracle.energy_forces(b, d, p, nl)
    assert np.allclose(out["E"], ref["E"], rtol=1e-14) and np.all(out["E_std"] <= 1e-12 * np.abs(ref["E"]))
    assert np.all(out["F_std"] <= 1e-12)
    a = oracle.energy_forces_ensemble(b, d, pe, nl, virial=False)
    perm = [2, 0, 1]
    pp = dict(pe, w3=np.asarray(pe["w3"])[:, perm].copy(), b3=np.asarray(pe["b3"])[perm].copy())
    c = oracle.energy_forces_ensemble(b, d, pp, nl, virial=False)
    assert np.allclose(a["E"], c["E"], rtol=1e-14) and np.allclose(a["E_std"], c["E_std"], rtol=1e-12)
    assert np.allclose(a["F_std"], c["F_std"], rtol=1e-10)
