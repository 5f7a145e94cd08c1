"""GPU parity of the Bessel-like radial basis and of the shallow-ensemble readout against the
FP64 oracle, through the C ABI (tolerances as for the Gaussian single-head model: FP32 1e-5,
mixed 2e-3)."""
import numpy as np
import pytest

import oracle
import synth
from synth.params import make_params
from tests.parity import ELEMENT_FACTOR, TOL, energy_error, force_error, subset, virial_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_22168_b300 import build
    build.build()


def _case(name):
    if name == "config1":
        return synth.config(1, activation="tanh")
    b, d, p = synth.config(3)
    return subset(b, range(24)), d, p


_REF = {}


def _ref(key, fn):
    if key not in _REF:
        _REF[key] = fn()
    return _REF[key]


# ------------------------------------------------------------------ Bessel-like basis

@pytest.mark.parametrize("precision", ["fp32", "mixed"])
@pytest.mark.parametrize("tpa", [0, 1, 8, 32])
@pytest.mark.parametrize("case", ["config1", "li_small"])
def test_bessel_basis_energy_forces_virial(case, tpa, precision):
    from paper_2505_22168_b300 import GMNN, DeviceSystem
    b, d, p = _case(case)
    d = dict(d, basis="bessel")
    ref = _ref(("bessel", case), lambda: oracle.energy_forces(b, d, p, oracle.neighbors(b, d["r_cut"])))
    m = GMNN(d, p, precision=precision)
    if tpa:
        m.set_tuning(pair_tpa=tpa)
    sysd = DeviceSystem(b)
    nl = m.build_neighbors(sysd)
    E, F, W = m.energy_forces(sysd, nl, virial=True)
    m.check_status()
    tol = TOL[precision]
    e = energy_error(E.cpu().numpy(), ref, b)
    f_rms, f_max = force_error(F.cpu().numpy().astype(np.float64), ref)
    assert e <= tol and f_rms <= tol and f_max <= ELEMENT_FACTOR * tol, (e, f_rms, f_max)
    assert virial_error(W.cpu().numpy(), ref) <= tol


def test_bessel_basis_descriptors():
    from paper_2505_22168_b300 import GMNN, DeviceSystem
    b, d, p = _case("config1")
    d = dict(d, basis="bessel")
    m = GMNN(d, p)
    sysd = DeviceSystem(b)
    nl = m.build_neighbors(sysd)
    psi, G = m.descriptors(sysd, nl)
    m.check_status()
    ref = oracle.energy_forces(b, d, p, oracle.neighbors(b, d["r_cut"]), psi=True, features=True)
    assert np.abs(psi.cpu().numpy() - ref["psi"]).max() <= 1e-5 * np.abs(ref["psi"]).max()
    assert np.abs(G.cpu().numpy() - ref["G"]).max() <= 1e-5 * np.abs(ref["G"]).max()


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_bessel_basis_param_grad(precision):
    """The parameter gradient with the Bessel basis (its beta gradient and the pair kernels'
    tangent moments use the basis) against the oracle's."""
    from paper_2505_22168_b300 import GMNN, DeviceSystem, unpack_theta
    b, d, p = _case("config1")
    d = dict(d, basis="bessel")
    onl = oracle.neighbors(b, d["r_cut"])
    ref = oracle.energy_forces(b, d, p, onl)
    rng = np.random.default_rng(4)
    _, gE, gF = oracle.loss(b, ref["E"], ref["E"] + rng.normal(0, 0.5, 1), ref["F"],
                            ref["F"] + rng.normal(0, 0.1, ref["F"].shape))
    go = oracle.param_grad(b, d, p, onl, gE, gF.astype(np.float32).astype(np.float64))
    m = GMNN(d, p, precision=precision)
    sysd = DeviceSystem(b)
    nl = m.build_neighbors(sysd)
    g = m.param_grad(sysd, nl, torch.as_tensor(gE, device=m.device), torch.as_tensor(gF, dtype=torch.float32,
                                                                                      device=m.device))
    m.check_status()
    gg = unpack_theta(g.cpu().numpy().astype(np.float64), d["n_species"], d["n_hidden"])
    tol = {"fp32": 1e-4, "mixed": 5e-3}[precision]
    for k in go:
        rel = np.linalg.norm(gg[k].ravel() - go[k].ravel()) / np.linalg.norm(go[k].ravel())
        assert rel <= tol, (k, rel)


# ------------------------------------------------------------------ shallow ensemble

N_HEADS = 4


def _ens_params(d, p):
    pe = make_params(d["n_species"], d["n_hidden"], 4242, 40.0, n_ensemble=N_HEADS)
    return dict(p, w3=pe["w3"], b3=pe["b3"])


def _ens_check(out, ref, b, precision, jac):
    tol = TOL[precision]
    Eh = out["E_heads"].cpu().numpy()
    # mean energy and the gradient of the mean energy (Eq. jacobian)
    assert energy_error(out["E"].cpu().numpy(), {"E": ref["E"], "E_atom": ref["E_atom"]}, b) <= tol
    f_rms, f_max = force_error(out["F"].cpu().numpy().astype(np.float64), ref)
    assert f_rms <= tol and f_max <= ELEMENT_FACTOR * tol, (f_rms, f_max)
    # every head's energy, and the spread (a 1-Lipschitz function of the head energies)
    worst = 0.0
    for k in range(N_HEADS):
        worst = max(worst, np.abs(Eh[:, k] - ref["E_heads"][:, k]).max())
        e = energy_error(Eh[:, k], {"E": ref["E_heads"][:, k], "E_atom": ref["E_atom"]}, b)
        assert e <= tol, (k, e)
    assert np.abs(out["E_std"].cpu().numpy() - ref["E_std"]).max() <= worst * (1 + 1e-9) + 1e-12
    assert ref["E_std"].min() > 10 * worst             # the spread is resolved, not noise
    if jac:
        Fh = out["F_heads"].cpu().numpy().astype(np.float64)
        dmax = np.zeros(b.n_atoms)
        for k in range(N_HEADS):
            r = {"F": ref["F_heads"][k]}
            f_rms, f_max = force_error(Fh[k], r)
            assert f_rms <= tol and f_max <= ELEMENT_FACTOR * tol, (k, f_rms, f_max)
            dmax = np.maximum(dmax, np.linalg.norm(Fh[k] - ref["F_heads"][k], axis=1))
        # the head mean equals the mean-gradient force (Eq. jacobian), up to rounding
        rms = np.sqrt((ref["F"] ** 2).mean())
        assert np.abs(Fh.mean(0) - out["F"].cpu().numpy()).max() <= ELEMENT_FACTOR * tol * rms
        Fs = out["F_std"].cpu().numpy().astype(np.float64)
        assert np.all(np.abs(Fs - ref["F_std"]) <= dmax * (1 + 1e-6) + 1e-6 * rms)


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
@pytest.mark.parametrize("mode", ["mean", "jacobian"])
@pytest.mark.parametrize("case", ["config1", "li_small"])
def test_shallow_ensemble_matches_oracle(case, mode, precision):
    from paper_2505_22168_b300 import GMNN, DeviceSystem
    b, d, p = _case(case)
    d = dict(d, n_ensemble=N_HEADS)
    pe = _ens_params(d, p)
    ref = _ref(("ens", case), lambda: oracle.energy_forces_ensemble(b, d, pe, oracle.neighbors(b, d["r_cut"])))
    m = GMNN(d, pe, precision=precision)
    sysd = DeviceSystem(b)
    nl = m.build_neighbors(sysd)
    out = m.energy_forces_ensemble(sysd, nl, mode=mode, virial=True)
    m.check_status()
    _ens_check(out, ref, b, precision, mode == "jacobian")
    assert virial_error(out["W"].cpu().numpy(), ref) <= TOL[precision]
    # the plain entry point on an ensemble model: the mean energy and its gradient
    E, F, _ = m.energy_forces(sysd, nl)
    m.check_status()
    assert energy_error(E.cpu().numpy(), {"E": ref["E"], "E_atom": ref["E_atom"]}, b) <= TOL[precision]
    assert force_error(F.cpu().numpy().astype(np.float64), ref)[0] <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
@pytest.mark.parametrize("n_boxes", [16, 34])
def test_shallow_ensemble_jacobian_head_chunks(n_boxes, precision):
    """The Jacobian mode stacks the backward passes of as many heads as keep heads x atoms
    within 16,384: 16 random-packed Li3PO4-like boxes of 512 atoms (8,192 atoms) run the four
    heads in two chunks of two, 34 boxes (17,408 atoms) one head at a time in the single-head
    buffers.  Against the oracle: every head's forces, the mean and the spreads."""
    from synth.systems import li3po4_random, make_batch
    from paper_2505_22168_b300 import GMNN, DeviceSystem
    _, d, p = synth.config(3)
    b = make_batch([li3po4_random(64, 7300 + k) for k in range(n_boxes)], 3)
    d = dict(d, n_ensemble=N_HEADS)
    pe = _ens_params(d, p)
    ref = _ref(("ens_chunks", n_boxes),
               lambda: oracle.energy_forces_ensemble(b, d, pe, oracle.neighbors(b, d["r_cut"]), virial=False))
    m = GMNN(d, pe, precision=precision)
    sysd = DeviceSystem(b)
    nl = m.build_neighbors(sysd)
    out = m.energy_forces_ensemble(sysd, nl, mode="jacobian")
    m.check_status()
    _ens_check(out, ref, b, precision, True)


def test_shallow_ensemble_rejects_what_it_does_not_support():
    from paper_2505_22168_b300 import GMNN, DeviceSystem, _lib
    b, d, p = _case("config1")
    m1 = GMNN(d, p)
    sysd = DeviceSystem(b)
    nl = m1.build_neighbors(sysd)
    with pytest.raises(_lib.GmError) as e:                  # one head: not an ensemble
        m1.energy_forces_ensemble(sysd, nl)
    assert e.value.code == _lib.GM_ERR_ARG
    d4 = dict(d, n_ensemble=N_HEADS)
    m4 = GMNN(d4, _ens_params(d4, p))
    with pytest.raises(_lib.GmError) as e:                  # no parameter gradient for ensembles
        m4.param_grad(sysd, nl, torch.zeros(1, dtype=torch.float64, device=m4.device),
                      torch.zeros(b.n_atoms, 3, dtype=torch.float32, device=m4.device))
    assert e.value.code == _lib.GM_ERR_UNSUPPORTED
