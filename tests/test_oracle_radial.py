"""CPU pins of the oracle's radial part: basis, cutoff and species-pair radial functions.

Section "Machine Learning Interatomic Potentials" of the paper names equidistant Gaussians
combined by element-pair coefficients into the radial functions R (Eq. basis_fn) but
prints no formula; the readings are Phi_k(r) = exp(-gamma (r - mu_k)^2) with
mu_k = r_min + k (r_c - r_min)/(n_b - 1), gamma = n_b^2 / r_c^2, the cosine cutoff
f_c(r) = (cos(pi r / r_c) + 1)/2 and R_s = f_c n_b^{-1/2} sum_k beta[Zi][Zj][s][k] Phi_k.
These tests hold the oracle to those readings with every constant written out as a
number (the centres, the width, the normalisation, exact cosine values), so that a wrong
width, a shifted or respaced centre, a missing normalisation or a transposed species pair
fails.
"""
import math

import numpy as np
import pytest

import oracle
from synth.params import make_params
from synth.systems import dimer, make_batch

# r_c = 5, n_b = 7, r_min = 0.5: centres every 0.75 A and gamma = 49/25
DESC = {"n_species": 2, "n_hidden": 64, "r_cut": 5.0, "r_min": 0.5, "n_basis": 7, "n_radial": 5,
        "activation": "tanh"}
MU = [0.5, 1.25, 2.0, 2.75, 3.5, 4.25, 5.0]
GAMMA = 1.96
INV_SQRT_NB = 0.3779644730092272          # 7^(-1/2)


@pytest.fixture(scope="module")
def params():
    p = make_params(2, 64, 77, 40.0)
    rng = np.random.default_rng(5)
    p["beta"] = rng.normal(0.0, 1.0, p["beta"].shape)     # beta[0][1] differs from beta[1][0]
    return p


# (r, f_c(r)) with exact cosines: cos(pi/3) = 1/2, cos(pi/2) = 0, cos(2 pi/3) = -1/2,
# cos(2 pi/5) = (sqrt 5 - 1)/4
CUTOFF_POINTS = [(0.0, 1.0), (5.0 / 3.0, 0.75), (2.0, 0.6545084971874737), (2.5, 0.5), (10.0 / 3.0, 0.25)]


@pytest.mark.parametrize("r,fc", CUTOFF_POINTS)
def test_gaussian_basis_times_cutoff_closed_form(params, r, fc):
    B, _ = oracle.radial_basis(DESC, params, r)
    want = np.array([fc * math.exp(-GAMMA * (r - m) ** 2) for m in MU])
    assert np.allclose(B, want, rtol=1e-13, atol=1e-300)


def test_basis_values_at_two_hand_computed_points(params):
    """Two entries computed by hand: at r = 2 the third Gaussian is centred (Phi = 1), and at
    r = 2.5 the cutoff is exactly 1/2 and the second Gaussian is exp(-1.96 * 1.5625)."""
    B, _ = oracle.radial_basis(DESC, params, 2.0)
    assert B[2] == pytest.approx(0.6545084971874737, rel=1e-14)
    B, _ = oracle.radial_basis(DESC, params, 2.5)
    assert B[1] == pytest.approx(0.5 * 0.04677062238395898, rel=1e-13)


def test_basis_derivative_matches_central_differences(params):
    h = 1e-6
    for r in (0.3, 1.1, 2.6, 4.2, 4.97):
        _, dB = oracle.radial_basis(DESC, params, r)
        Bp, _ = oracle.radial_basis(DESC, params, r + h)
        Bm, _ = oracle.radial_basis(DESC, params, r - h)
        assert np.allclose(dB, (Bp - Bm) / (2 * h), rtol=1e-7, atol=1e-9), r


def test_cutoff_and_its_slope_vanish_at_r_cut(params):
    """f_c(r_c) = f_c'(r_c) = 0: the basis and its derivative are zero at and beyond r_c and
    go to zero as (r_c - r)^2 and (r_c - r) below it."""
    for r in (5.0, 5.3):
        B, dB = oracle.radial_basis(DESC, params, r)
        assert np.all(B == 0.0) and np.all(dB == 0.0)
    for h in (1e-2, 1e-3):
        B, dB = oracle.radial_basis(DESC, params, 5.0 - h)
        # f_c(r_c - h) = (1 - cos(pi h / r_c))/2 ~ (pi h / r_c)^2 / 4; Phi_k <= 1
        assert np.abs(B).max() <= 1.01 * (math.pi * h / 5.0) ** 2 / 4
        assert np.abs(dB).max() <= 1.01 * (math.pi / 5.0) ** 2 * h / 2 + 2 * GAMMA * 4.5 * (math.pi * h / 5.0) ** 2 / 4


def _radial_by_hand(beta, zi, zj, r, fc):
    phi = np.array([math.exp(-GAMMA * (r - m) ** 2) for m in MU])
    return INV_SQRT_NB * fc * (beta[zi, zj] @ phi)


@pytest.mark.parametrize("r,fc", CUTOFF_POINTS[1:])
def test_radial_functions_use_the_ordered_species_pair(params, r, fc):
    beta = np.asarray(params["beta"])
    R01, _ = oracle.radial_fns(DESC, params, 0, 1, r)
    R10, _ = oracle.radial_fns(DESC, params, 1, 0, r)
    assert np.allclose(R01, _radial_by_hand(beta, 0, 1, r, fc), rtol=1e-12, atol=1e-15)
    assert np.allclose(R10, _radial_by_hand(beta, 1, 0, r, fc), rtol=1e-12, atol=1e-15)
    assert np.abs(R01 - R10).max() > 1e-3 * np.abs(R01).max()     # the pair order matters


@pytest.mark.parametrize("r,fc", [(2.0, 0.6545084971874737), (2.5, 0.5), (10.0 / 3.0, 0.25)])
def test_dimer_rank0_moments_are_the_radial_functions(params, r, fc):
    """Through the full model: a dimer of species 0 and 1 has Psi_{i,0,s} = R_{Zi,Zj,s}(r)
    (one neighbour, rhat^0 = 1).  Atom 0 must carry beta[0][1], atom 1 beta[1][0]."""
    pos, spec, cell = dimer(r, direction=(0.3, -0.5, 0.8), species=(0, 1), box=40.0)
    b = make_batch([(pos, spec, cell)], 2)
    nl = oracle.neighbors(b, DESC["r_cut"])
    out = oracle.energy_forces(b, DESC, params, nl, psi=True)
    beta = np.asarray(params["beta"])
    psi0 = out["psi"][:, :, 0]
    assert np.allclose(psi0[0], _radial_by_hand(beta, 0, 1, r, fc), rtol=1e-12, atol=1e-15)
    assert np.allclose(psi0[1], _radial_by_hand(beta, 1, 0, r, fc), rtol=1e-12, atol=1e-15)
    swapped = _radial_by_hand(beta, 1, 0, r, fc)
    assert np.abs(psi0[0] - swapped).max() > 1e-3 * np.abs(psi0[0]).max()


# ----------------------------------------------------------------- Bessel-like basis
# The second basis the paper names (Kocer et al.): f_k = a_k [j0((k+1) pi r/r_c) +
# j0((k+2) pi r/r_c)].  The zeroth-order spherical Bessel functions j0(n pi r / r_c) are
# orthogonal on [0, r_c] with weight r^2 (norm r_c^3 / (2 n^2 pi^2)), so the f_k are unit
# vectors, f_k and f_(k+1) share one term (overlap of sign -1), and f_k, f_l with |k - l| >= 2
# are orthogonal.  Each f_k and its slope vanish at r_c.  These properties come from the
# mathematics of j0, not from the formula typed again.

BESSEL = dict(DESC, basis="bessel")


def _bessel_only(params, r):
    """f_k(r) without the cutoff: the oracle's f_c f_k divided by f_c (pinned above)."""
    B, dB = oracle.radial_basis(BESSEL, params, r)
    fc = 0.5 * (math.cos(math.pi * r / 5.0) + 1.0)
    return B / fc


def test_bessel_basis_is_orthonormal_with_weight_r_squared(params):
    x, w = np.polynomial.legendre.leggauss(400)
    r = 2.5 * (x + 1.0)                       # [0, 5]
    w = 2.5 * w
    F = np.array([_bessel_only(params, ri) for ri in r])          # [nodes, 7]
    gram = (F * (w * r * r)[:, None]).T @ F
    assert np.allclose(np.diag(gram), 1.0, atol=1e-9)
    for k in range(7):
        for l in range(7):
            if abs(k - l) >= 2:
                assert abs(gram[k, l]) <= 1e-9, (k, l)
            elif abs(k - l) == 1:
                assert gram[k, l] < -1e-3, (k, l)    # one shared term, opposite signs


def test_bessel_basis_and_slope_vanish_at_r_cut(params):
    B, dB = oracle.radial_basis(BESSEL, params, 5.0)
    assert np.all(B == 0.0) and np.all(dB == 0.0)
    f1 = np.abs(_bessel_only(params, 5.0 - 1e-2))
    f2 = np.abs(_bessel_only(params, 5.0 - 1e-3))
    # f_k(r_c - h) = O(h^2): ten times closer, about a hundred times smaller
    assert np.all(f2 <= 0.02 * f1 + 1e-12) and np.all(f1 < 2e-2)


def test_bessel_basis_derivative_matches_central_differences(params):
    h = 1e-6
    for r in (0.4, 1.3, 2.6, 3.9, 4.95):
        _, dB = oracle.radial_basis(BESSEL, params, r)
        Bp, _ = oracle.radial_basis(BESSEL, params, r + h)
        Bm, _ = oracle.radial_basis(BESSEL, params, r - h)
        assert np.allclose(dB, (Bp - Bm) / (2 * h), rtol=1e-7, atol=1e-9), r


def test_bessel_model_forces_and_virial_match_autograd_and_differences():
    import synth
    from oracle import torch_ref
    b, d, p = synth.config(1, activation="tanh")
    d = dict(d, basis="bessel")
    nl = oracle.neighbors(b, d["r_cut"])
    out = oracle.energy_forces(b, d, p, nl)
    t = torch_ref.energy_forces(b, d, p, nl)
    assert abs(out["E"][0] - t["E"][0]) <= 1e-12 * np.abs(t["E_atom"]).sum()
    assert np.abs(out["F"] - t["F"]).max() <= 1e-12 * np.abs(t["F"]).max()
    assert np.abs(out["virial"] - t["virial"]).max() <= 1e-12 * np.abs(t["virial"]).max()
    # central differences of the energy for a few atoms
    h = 1e-5
    for k in (0, 40, 95):
        for c in range(3):
            e = []
            for sgn in (1, -1):
                pos = b.pos.copy()
                pos[k, c] += sgn * h
                b2 = make_batch([(pos, b.species, b.cell[0])], b.n_species)
                e.append(oracle.energy_forces(b2, d, p, nl, virial=False)["E"][0])
            fd = -(e[0] - e[1]) / (2 * h)
            assert abs(fd - out["F"][k, c]) <= 1e-6 * np.abs(out["F"]).max(), (k, c)
    # the Bessel model is a different function of the positions than the Gaussian one
    g = oracle.energy_forces(b, dict(d, basis="gaussian"), p, nl)
    assert np.abs(g["F"] - out["F"]).max() > 1e-2 * np.abs(out["F"]).max()
