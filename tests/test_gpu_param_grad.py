"""GPU force-matching loss and parameter gradient (force double-backward) against the FP64
oracle, through the C ABI and through the torch.autograd.Function.

Tolerance (the paper states none for the gradient): relative L2 error per parameter group
<= 1e-4 for the FP32 kernels, and element-wise |error| <= 1e-3 x max|group|.  The mixed path
(network GEMMs on tcgen05 with BF16 operands and FP32 accumulation; by default all four GEMMs
of the parameter gradient run with hi/lo split operands) is held to 5e-3 relative L2 per group
and 5e-3 element-wise of the group's largest entry."""
import numpy as np
import pytest

import oracle
import synth
from tests.parity import energy_error, subset

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GROUPS = ("beta", "W1", "b1", "W2", "b2", "w3", "b3", "sigma", "mu")
TOL_L2 = {"fp32": 1e-4, "mixed": 5e-3}
TOL_ELEM = {"fp32": 1e-3, "mixed": 5e-3}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_22168_b300 import build
    build.build()


def _setup(batch, desc, params, precision="fp32", seed=11):
    from paper_2505_22168_b300 import GMNN, DeviceSystem
    m = GMNN(desc, params, precision=precision)
    sysd = DeviceSystem(batch)
    nl = m.build_neighbors(sysd)
    onl = oracle.neighbors(batch, desc["r_cut"])
    ref = oracle.energy_forces(batch, desc, params, onl)
    rng = np.random.default_rng(seed)
    Eref = ref["E"] + rng.normal(0, 0.5, ref["E"].shape)
    Fref = ref["F"] + rng.normal(0, 0.1, ref["F"].shape)
    return m, sysd, nl, onl, ref, Eref, Fref


def _compare(g_dev, go, n_species, n_hidden, precision="fp32"):
    from paper_2505_22168_b300 import unpack_theta
    g = unpack_theta(g_dev.cpu().numpy().astype(np.float64), n_species, n_hidden)
    worst = {}
    for k in GROUPS:
        ref = go[k].reshape(-1)
        got = g[k].reshape(-1)
        scale = np.linalg.norm(ref)
        assert scale > 0, k
        rel = np.linalg.norm(got - ref) / scale
        elem = np.abs(got - ref).max() / np.abs(ref).max()
        worst[k] = (rel, elem)
        assert rel <= TOL_L2[precision], (k, rel)
        assert elem <= TOL_ELEM[precision], (k, elem)
    return worst


def _param_grad_case(batch, desc, params, precision="fp32"):
    m, sysd, nl, onl, ref, Eref, Fref = _setup(batch, desc, params, precision=precision)
    E, F, _ = m.energy_forces(sysd, nl)
    m.check_status()
    # the loss kernel, on the GPU's own energies and forces
    Eref_d = torch.as_tensor(Eref, device=m.device)
    Fref_d = torch.as_tensor(Fref, dtype=torch.float32, device=m.device)
    loss, gE, gF = m.force_matching_loss(sysd, E, Eref_d, F, Fref_d)
    L_g, gE_g, gF_g = oracle.loss(batch, E.cpu().numpy(), Eref, F.cpu().numpy().astype(np.float64),
                                  Fref_d.cpu().numpy().astype(np.float64))
    assert abs(float(loss.item()) - L_g) <= 1e-12 * abs(L_g)
    assert np.abs(gE.cpu().numpy() - gE_g).max() <= 1e-12 * np.abs(gE_g).max()
    assert np.abs(gF.cpu().numpy() - gF_g).max() <= 1e-6 * np.abs(gF_g).max()
    # the parameter gradient, with the oracle's dL/dE and dL/dF fed to both sides
    _, gE_o, gF_o = oracle.loss(batch, ref["E"], Eref, ref["F"], Fref)
    g = m.param_grad(sysd, nl, torch.as_tensor(gE_o, device=m.device),
                     torch.as_tensor(gF_o, dtype=torch.float32, device=m.device))
    m.check_status()
    go = oracle.param_grad(batch, desc, params, onl, gE_o, gF_o.astype(np.float32).astype(np.float64))
    return _compare(g, go, desc["n_species"], desc["n_hidden"], precision)


@pytest.mark.parametrize("act", ["tanh", "silu"])
def test_param_grad_config1(act):
    b, d, p = synth.config(1, activation=act)
    _param_grad_case(b, d, p)


def test_param_grad_emim_batch():
    """Several EMIM boxes of different sizes (the training workload's structure)."""
    b4, d, p = synth.config(4)
    _param_grad_case(subset(b4, [0, 1, 2, 5]), d, p)


@pytest.mark.parametrize("act", ["tanh", "silu"])
def test_param_grad_mixed_precision(act):
    """BF16 network GEMMs on tcgen05 in the parameter gradient (training with a BF16 MLP)."""
    b4, d, p = synth.config(4, activation=act)
    worst = _param_grad_case(subset(b4, [0, 1, 2, 5]), d, p, precision="mixed")
    print("mixed param-grad errors (rel L2, elementwise):", {k: tuple(round(x, 6) for x in v) for k, v in worst.items()})


def test_param_grad_small_li3po4_boxes_multi_image():
    b3, d, p = synth.config(3)
    p = dict(p)
    _param_grad_case(subset(b3, range(6)), d, p)


def test_autograd_function_backward_matches_oracle():
    """theta.grad from loss.backward() through GMNNFunction equals the oracle's gradient of
    the same loss (computed here with torch ops on the outputs)."""
    from paper_2505_22168_b300 import GMNNFunction, pack_theta
    b, d, p = synth.config(1, activation="silu")
    m, sysd, nl, onl, ref, Eref, Fref = _setup(b, d, p)
    theta = torch.as_tensor(pack_theta(p), device=m.device).requires_grad_(True)
    E, F = GMNNFunction.apply(theta, m, sysd, nl)
    nat = torch.as_tensor(np.diff(b.atom_ptr), dtype=torch.float64, device=m.device)
    L = (((E - torch.as_tensor(Eref, device=m.device)) / nat) ** 2).mean() + \
        ((F.double() - torch.as_tensor(Fref, device=m.device)) ** 2).sum() / (3 * b.n_atoms)
    L.backward()
    m.check_status()
    # the oracle's gradient of the same loss at the same (GPU) energies and forces
    _, gE_o, gF_o = oracle.loss(b, E.detach().cpu().numpy(), Eref, F.detach().cpu().numpy().astype(np.float64), Fref)
    go = oracle.param_grad(b, d, p, onl, gE_o, gF_o)
    _compare(theta.grad, go, d["n_species"], d["n_hidden"])


@pytest.mark.parametrize("tpa", [1, 2, 4, 8, 16, 32])
def test_param_grad_every_pair_lane_count(tpa):
    """The parameter gradient's pair kernels (moments, tangent moments, the beta gradient) at
    every lanes-per-atom setting, FP32, on the 96-atom box."""
    b, d, p = synth.config(1, activation="tanh")
    m, sysd, nl, onl, ref, Eref, Fref = _setup(b, d, p)
    m.set_tuning(pair_tpa=tpa)
    _, gE_o, gF_o = oracle.loss(b, ref["E"], Eref, ref["F"], Fref)
    g = m.param_grad(sysd, nl, torch.as_tensor(gE_o, device=m.device),
                     torch.as_tensor(gF_o, dtype=torch.float32, device=m.device))
    m.check_status()
    go = oracle.param_grad(b, d, p, onl, gE_o, gF_o.astype(np.float32).astype(np.float64))
    _compare(g, go, d["n_species"], d["n_hidden"])


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_autograd_training_steps_follow_the_updated_weights(precision):
    """Three optimiser steps through GMNNFunction.  The optimiser updates theta in place, so
    every forward must use the updated weights: after each step the energies, forces and
    theta.grad equal the oracle's at the current theta."""
    from paper_2505_22168_b300 import GMNNFunction, pack_theta, unpack_theta
    b4, d, p = synth.config(4, activation="silu")
    b = subset(b4, [0, 2])
    m, sysd, nl, onl, ref, Eref, Fref = _setup(b, d, p, precision=precision)
    theta = torch.as_tensor(pack_theta(p), device=m.device).requires_grad_(True)
    opt = torch.optim.SGD([theta], lr=0.05)
    nat = torch.as_tensor(np.diff(b.atom_ptr), dtype=torch.float64, device=m.device)
    Eref_d = torch.as_tensor(Eref, device=m.device)
    Fref_d = torch.as_tensor(Fref, device=m.device)
    tol_f = {"fp32": 1e-5, "mixed": 2e-3}[precision]
    last = None
    for step in range(3):
        opt.zero_grad()
        E, F = GMNNFunction.apply(theta, m, sysd, nl)
        L = (((E - Eref_d) / nat) ** 2).mean() + ((F.double() - Fref_d) ** 2).sum() / (3 * b.n_atoms)
        L.backward()
        m.check_status()
        cur = unpack_theta(theta.detach().cpu().numpy().astype(np.float64), d["n_species"], d["n_hidden"])
        r = oracle.energy_forces(b, d, cur, onl, virial=False)
        Fg = F.detach().cpu().numpy().astype(np.float64)
        rms = np.sqrt((r["F"] ** 2).mean())
        assert np.sqrt(((Fg - r["F"]) ** 2).mean()) / rms <= tol_f, step
        Eg = E.detach().cpu().numpy()
        assert energy_error(Eg, r, b) <= tol_f, step
        _, gE_o, gF_o = oracle.loss(b, Eg, Eref, Fg, Fref)
        go = oracle.param_grad(b, d, cur, onl, gE_o, gF_o)
        _compare(theta.grad, go, d["n_species"], d["n_hidden"], precision)
        if last is not None:
            assert not np.array_equal(Fg, last)          # the weights did change
        last = Fg
        opt.step()
