"""The network as one tcgen05 kernel with each 128-atom tile split over a thread-block
cluster (2, 4 or 8 CTAs along the hidden width, the layer activations all-gathered between
layers): parity with the FP64 oracle and with the one-CTA-per-tile kernel.

Both fused kernels round the same operands the same way (BF16 forward, FP16 backward, phi'
kept in FP16) and accumulate every output element over the same K blocks in the same order,
so their output-layer partial sums, and with them the energies (fixed-point sums of the same
per-atom values), agree bit for bit; forces agree up to the order of their FP32 atomic sums."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from synth.systems import make_batch
from tests.parity import ELEMENT_FACTOR, TOL, energy_error, force_error, subset, virial_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2505_22168_b300 import build
    build.build()


def _gm():
    from paper_2505_22168_b300 import GMNN, DeviceSystem
    return GMNN, DeviceSystem


def _case(name):
    """(batch, desc, params): widths 128 (96 atoms), 512 (1536 atoms, and a two-structure
    1700-atom batch whose tiles end ragged and straddle a structure boundary) and 256 (24
    Li3PO4-like boxes of different sizes)."""
    if name == "config1":
        return synth.config(1)
    if name == "config2":
        return synth.config(2)
    if name == "config2_ragged":
        b, d, p = synth.config(2)
        s = [(b.pos[:1400], b.species[:1400], b.cell[0]), (b.pos[:300], b.species[:300], b.cell[0])]
        return make_batch(s, b.n_species), d, p
    b, d, p = synth.config(3)
    return subset(b, range(24)), d, p


CASES = [("config1", 2), ("config2", 2), ("config2", 4), ("config2", 8), ("config2_ragged", 8),
         ("config2_ragged", 4), ("li_small", 2), ("li_small", 4)]


def _run(b, d, p, cs, virial):
    GMNN, DeviceSystem = _gm()
    sysd = DeviceSystem(b)
    mm = GMNN(d, p, precision="mixed")
    nl = mm.build_neighbors(sysd)
    mm.set_tuning(fused_mlp=1, mlp_cluster=cs)
    out = mm.energy_forces(sysd, nl, virial=virial)
    mm.check_status()
    return [None if x is None else x.cpu().numpy() for x in out]


@pytest.mark.parametrize("case,cs", CASES)
def test_cluster_network_kernel_matches_oracle_and_per_tile_kernel(case, cs):
    b, d, p = _case(case)
    ref = oracle.energy_forces(b, d, p, oracle.neighbors(b, d["r_cut"]))
    tol = TOL["mixed"]
    # energies summed inside the cluster kernel (no virial)
    E, F, _ = _run(b, d, p, cs, virial=False)
    e = energy_error(E, ref, b)
    f_rms, f_max = force_error(F.astype(np.float64), ref)
    assert e <= tol and f_rms <= tol and f_max <= ELEMENT_FACTOR * tol, (e, f_rms, f_max)
    # with the virial: energies and virials from the reduction kernel
    Ev, Fv, Wv = _run(b, d, p, cs, virial=True)
    assert np.array_equal(E, Ev)
    assert virial_error(Wv, ref) <= tol
    # the one-CTA-per-tile kernel: same energies bit for bit, forces up to atomic order
    E1, F1, _ = _run(b, d, p, 1, virial=False)
    assert np.array_equal(E, E1)
    assert np.abs(F - F1).max() <= 1e-5 * np.abs(F1).max()


@pytest.mark.parametrize("act", ["tanh", "silu"])
def test_cluster_network_kernel_both_activations(act):
    b, d, p = synth.config(2, activation=act)
    ref = oracle.energy_forces(b, d, p, oracle.neighbors(b, d["r_cut"]))
    E, F, _ = _run(b, d, p, 8, virial=False)
    tol = TOL["mixed"]
    e = energy_error(E, ref, b)
    f_rms, f_max = force_error(F.astype(np.float64), ref)
    assert e <= tol and f_rms <= tol and f_max <= ELEMENT_FACTOR * tol, (e, f_rms, f_max)


def test_cluster_form_by_size_replays_in_a_graph():
    """The default (by size) form at 1536 atoms, replayed as a CUDA graph of the whole step
    with moved positions: each replay equals a direct call on the same positions (energies bit
    for bit, forces up to atomic order)."""
    GMNN, DeviceSystem = _gm()
    b, d, p = synth.config(2)
    sysd = DeviceSystem(b)
    mm = GMNN(d, p, precision="mixed")
    nl = mm.build_neighbors(sysd)
    out = mm.energy_forces(sysd, nl)
    g = mm.capture_step(sysd, nl, out)
    rng = np.random.default_rng(5)
    for _ in range(3):
        pos = b.pos + rng.normal(0.0, 0.01, b.pos.shape)
        sysd.pos.copy_(torch.as_tensor(pos))
        g.replay()
        torch.cuda.synchronize()
        mm.check_status()
        E, F = out[0].cpu().numpy(), out[1].cpu().numpy()
        E2, F2, _ = mm.energy_forces(sysd, mm.build_neighbors(sysd))
        mm.check_status()
        assert np.array_equal(E, E2.cpu().numpy())
        assert np.abs(F - F2.cpu().numpy()).max() <= 1e-5 * np.abs(F).max()
