"""GPU parity against the FP64 oracle, through the C ABI.

Neighbour sets are compared bit for bit (as sorted (i, j, shift) triples).  Energies,
forces, virials and descriptors are compared element by element within the tolerance
stated for the FP32 path (1e-5 relative on energy per atom and force RMS).
"""
import dataclasses

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
        pytest.skip("no CUDA device")
    from paper_2505_22168_b300 import build
    build.build()


def _gm():
    from paper_2505_22168_b300 import GMNN, DeviceSystem
    return GMNN, DeviceSystem


def _model(desc, params, precision="fp32"):
    GMNN, _ = _gm()
    return GMNN(desc, params, precision=precision)


def _nl_pair(batch, desc, params):
    GMNN, DeviceSystem = _gm()
    m = GMNN(desc, params)
    sysd = DeviceSystem(batch)
    nl = m.build_neighbors(sysd)
    return m, sysd, nl


@pytest.fixture(scope="module")
def li_small():
    b, d, p = synth.config(3)
    return subset(b, range(24)), d, p


# ------------------------------------------------------------------ neighbour lists

def _assert_same_pairs(batch, desc, params):
    _, _, nl = _nl_pair(batch, desc, params)
    got = nl.triples()
    want = oracle.neighbors(batch, desc["r_cut"]).triples()
    assert got.shape == want.shape
    assert np.array_equal(got, want)
    assert int(nl.n_pairs.item()) == len(want)


def test_neighbors_config1():
    b, d, p = synth.config(1)
    _assert_same_pairs(b, d, p)


def test_neighbors_small_boxes_multi_image(li_small):
    b, d, p = li_small
    L = b.cell[:, 0, 0]
    assert (L < 2 * d["r_cut"]).any()          # several images of one neighbour occur
    _assert_same_pairs(b, d, p)


@pytest.mark.parametrize("rc,count", [(0.99, 0), (1.01, 6), (1.5, 18), (2.1, 32), (2.5, 80)])
def test_neighbors_self_images(rc, count):
    _, d, p = synth.config(1)
    d = dict(d, r_cut=rc, r_min=0.1)
    b = make_batch([(np.array([[0.3, 0.6, 0.9]]), np.array([0]), np.eye(3))], 5)
    _, _, nl = _nl_pair(b, d, p)
    assert int(nl.n_pairs.item()) == count
    assert np.array_equal(nl.triples(), oracle.neighbors(b, rc).triples())


def test_neighbors_outside_cell_ragged_and_empty():
    """Positions far outside the cell, structures of different sizes, and an empty one."""
    _, d, p = synth.config(1)
    _assert_same_pairs(_ragged_batch(), dict(d, r_cut=3.3), p)


def test_neighbors_exactly_at_cutoff():
    _, d, p = synth.config(1)
    pos = np.array([[1.0, 1.0, 1.0], [1.0 + 2.5, 1.0, 1.0], [1.0, 1.0 + np.nextafter(2.5, 0.0), 1.0]])
    b = make_batch([(pos, np.array([0, 1, 2]), 20 * np.eye(3))], 5)
    _assert_same_pairs(b, dict(d, r_cut=2.5, r_min=0.2), p)


# launch shapes of the neighbour build: one cooperative launch (default) or one launch per
# phase; blocks per home cell; grid size.  None of them may change the list or its order.
NL_TUNINGS = [dict(nl_mode=0), dict(nl_mode=1), dict(nl_mode=0, nl_split=1), dict(nl_mode=0, nl_split=3, nl_blocks=7),
              dict(nl_mode=1, nl_split=2), dict(nl_mode=0, nl_blocks=1), dict(nl_mode=0, nl_two_pass=1),
              dict(nl_mode=1, nl_two_pass=1, nl_split=5), dict(nl_items=1), dict(nl_items=2),
              dict(nl_items=1, nl_split=3, nl_two_pass=1), dict(nl_items=2, nl_split=3, nl_mode=1), dict(nl_items=3)]


def _ragged_batch():
    rng = np.random.default_rng(3)
    structs = []
    for L, n in ((4.0, 5), (7.0, 40), (9.0, 0), (5.5, 17), (12.0, 130)):
        structs.append((rng.uniform(-2 * L, 3 * L, (n, 3)), rng.integers(0, 5, n), L * np.eye(3)))
    return make_batch(structs, 5)


def _mid_size_li3po4():
    """Li3PO4-like boxes, some shorter than 2 r_cut, with 4096 < atoms + boxes <= 8192: the
    mid-size cooperative path, whose short boxes take the multi-image rows of the brute-force
    search."""
    b3, d, p = synth.config(3)
    k, n = 0, 0
    while n + k + 1 + (b3.atom_ptr[k + 1] - b3.atom_ptr[k]) <= 8000:
        n += b3.atom_ptr[k + 1] - b3.atom_ptr[k]
        k += 1
    b = subset(b3, range(k))
    assert 4096 < b.n_atoms + b.n_structures <= 8192
    assert (b.cell[:, 0, 0] < 2.001 * d["r_cut"]).any()
    return b, d, p


def _batch_li3po4(n_struct=40):
    """The first boxes of the Li3PO4-like batch, more than 8192 atoms + boxes (the general
    cooperative path), some boxes shorter than 2 r_cut (multi-image rows)."""
    b3, d, p = synth.config(3)
    b = subset(b3, range(n_struct))
    assert b.n_atoms + b.n_structures > 8192
    assert (b.cell[:, 0, 0] < 2.001 * d["r_cut"]).any()
    return b, d, p


@pytest.mark.parametrize("case", ["config1", "li_small", "config2", "ragged", "shifted", "train_batch",
                                  "mid_multi_image", "batch_multi_image"])
def test_neighbor_build_launch_shapes_give_identical_rows(case, li_small):
    """Every launch shape, the cell-list searches (nl_items 1, 2) included, gives the oracle's
    pairs in the same rows and order.  (train_batch: 32 EMIM boxes, 7920 atoms -- the mid-size
    path's brute-force search; mid_multi_image: the same path with multi-image rows;
    batch_multi_image: the brute-force search of the general path, multi-image rows.)"""
    GMNN, DeviceSystem = _gm()
    if case == "li_small":
        b, d, p = li_small
    elif case == "train_batch":
        b, d, p = synth.config(4)
        assert 4096 < b.n_atoms + b.n_structures <= 8192
        assert (b.cell[:, 0, 0] >= 2.001 * d["r_cut"]).all()
    elif case == "mid_multi_image":
        b, d, p = _mid_size_li3po4()
    elif case == "batch_multi_image":
        b, d, p = _batch_li3po4()
    elif case == "ragged":
        _, d, p = synth.config(1)
        b, d = _ragged_batch(), dict(d, r_cut=3.3)
    elif case == "shifted":            # every atom two boxes up along x, one down along z
        b, d, p = synth.config(2)
        L = b.cell[0].diagonal()
        b = dataclasses.replace(b, pos=b.pos + np.array([2.0 * L[0], 0.0, -L[2]]))
    else:
        b, d, p = synth.config(1 if case == "config1" else 2)
    want = oracle.neighbors(b, d["r_cut"]).triples()
    ref = None
    for tune in NL_TUNINGS:
        m = GMNN(d, p)
        m.set_tuning(**tune)
        nl = m.build_neighbors(DeviceSystem(b))
        assert np.array_equal(nl.triples(), want), tune
        P = int(nl.n_pairs.item())
        rows = (nl.row_ptr.cpu().numpy(), nl.col[:P].cpu().numpy(), nl.shift[:P].cpu().numpy())
        if ref is None:
            ref = rows
        else:
            assert all(np.array_equal(x, y) for x, y in zip(rows, ref)), tune


def test_neighbors_rows_longer_than_the_search_slab():
    """A dense ball in a sparse box: the ball's rows are far longer than the mean row the
    search slab is sized for, so the compaction searches them again."""
    GMNN, DeviceSystem = _gm()
    _, d, p = synth.config(1)
    rng = np.random.default_rng(11)
    L = 30.0
    ball = 15.0 + rng.normal(0.0, 1.0, (120, 3))
    sparse = rng.uniform(0.0, L, (600, 3))
    pos = np.concatenate([sparse[:300], ball, sparse[300:]])
    b = make_batch([(pos, rng.integers(0, 5, len(pos)), L * np.eye(3))], 5)
    want = oracle.neighbors(b, d["r_cut"])
    ref = None
    for tune in (dict(), dict(nl_two_pass=1), dict(nl_mode=1), dict(nl_items=1), dict(nl_items=2)):
        m = GMNN(d, p)
        m.set_tuning(**tune)
        nl = m.build_neighbors(DeviceSystem(b))
        got = nl.triples()
        assert np.array_equal(got, want.triples()), tune
        P = int(nl.n_pairs.item())
        cur = (nl.row_ptr.cpu().numpy(), nl.col[:P].cpu().numpy(), nl.shift[:P].cpu().numpy())
        if ref is None:
            ref = cur
            slab_row = max(64, -(-(nl.capacity * 3 // (2 * b.n_atoms) + 16) // 32) * 32)
            assert np.diff(cur[0]).max() > slab_row                   # some rows exceed the slab
        else:
            assert all(np.array_equal(x, y) for x, y in zip(cur, ref)), tune


def test_brute_force_rows_beyond_the_buffer_fall_back_to_cells():
    """A single-image box whose dense ball gives rows longer than the brute-force search's
    shared-memory buffer: the build switches to the cell list and still returns the oracle's
    pairs, in the same rows as an explicit cell-list build."""
    GMNN, DeviceSystem = _gm()
    _, d, p = synth.config(1)
    rng = np.random.default_rng(17)
    L = 40.0
    ball = 20.0 + rng.normal(0.0, 1.2, (700, 3))
    sparse = rng.uniform(0.0, L, (300, 3))
    pos = np.concatenate([sparse[:150], ball, sparse[150:]])
    b = make_batch([(pos, rng.integers(0, 5, len(pos)), L * np.eye(3))], 5)
    want = oracle.neighbors(b, d["r_cut"])
    assert np.diff(want.row_ptr).max() > 512
    rows = []
    for tune in (dict(), dict(nl_items=1)):
        m = GMNN(d, p)
        m.set_tuning(**tune)
        nl = m.build_neighbors(DeviceSystem(b))
        assert np.array_equal(nl.triples(), want.triples()), tune
        P = int(nl.n_pairs.item())
        rows.append((nl.row_ptr.cpu().numpy(), nl.col[:P].cpu().numpy(), nl.shift[:P].cpu().numpy()))
    assert all(np.array_equal(x, y) for x, y in zip(rows[0], rows[1]))


def test_neighbor_build_is_graph_capturable():
    """The cooperative build replays inside a CUDA graph and follows moved positions."""
    GMNN, DeviceSystem = _gm()
    b, d, p = synth.config(2)
    m = GMNN(d, p)
    sysd = DeviceSystem(b)
    nl = m.build_neighbors(sysd)
    from paper_2505_22168_b300 import NeighborList
    from paper_2505_22168_b300 import _lib
    from paper_2505_22168_b300.gmnn import _ptr, _stream
    nl2 = NeighborList(b.n_atoms, nl.capacity + 4096, m.device)
    ws, wsb = m.workspace(_lib.GM_OP_NEIGHBORS, sysd, nl2.capacity)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        _lib.gm_build_neighbors(m.handle, sysd.c_struct(), nl2.c_struct(), ws, wsb, _ptr(m.status), _stream())
    rng = np.random.default_rng(5)
    for step in range(3):
        moved = b.pos + rng.normal(0.0, 0.05, b.pos.shape)
        sysd.pos.copy_(torch.as_tensor(moved))
        m.clear_status()
        g.replay()
        torch.cuda.synchronize()
        assert m.read_status() == 0
        bm = dataclasses.replace(b, pos=moved)
        assert np.array_equal(nl2.triples(), oracle.neighbors(bm, d["r_cut"]).triples()), step


def test_neighbors_capacity_overflow_reports_required_count():
    from paper_2505_22168_b300 import NeighborList, _lib
    b, d, p = synth.config(1)
    m, sysd, _ = _nl_pair(b, d, p)
    small = NeighborList(sysd.n_atoms, 100, m.device)
    m.build_neighbors(sysd, small, check=False)
    assert m.read_status() == _lib.GM_ERR_CAPACITY
    assert int(small.n_pairs.item()) == oracle.neighbors(b, d["r_cut"]).n_pairs


def test_non_orthorhombic_cell_is_unsupported():
    from paper_2505_22168_b300 import _lib
    b, d, p = synth.config(1)
    cell = b.cell[0].copy()
    cell[1, 0] = 0.5
    b2 = make_batch([(b.pos, b.species, cell)], 5)
    GMNN, DeviceSystem = _gm()
    m = GMNN(d, p)
    m.build_neighbors(DeviceSystem(b2), check=False)
    assert m.read_status() == _lib.GM_ERR_UNSUPPORTED


def test_more_than_max_atoms_is_unsupported():
    """Checked on the host before anything touches the (much smaller) buffers."""
    from paper_2505_22168_b300 import _lib
    from paper_2505_22168_b300.gmnn import _ptr, _stream
    b, d, p = synth.config(1)
    m, sysd, nl = _nl_pair(b, d, p)
    c = sysd.c_struct()
    c.n_atoms = _lib.GM_MAX_ATOMS + 1
    ws, wsb = m.workspace(_lib.GM_OP_NEIGHBORS, sysd, nl.capacity)
    with pytest.raises(_lib.GmError) as err:
        _lib.gm_build_neighbors(m.handle, c, nl.c_struct(), ws, wsb, _ptr(m.status), _stream())
    assert err.value.code == _lib.GM_ERR_UNSUPPORTED


def test_bad_species_is_reported():
    from paper_2505_22168_b300 import _lib
    b, d, p = synth.config(1)
    spec = b.species.copy()
    spec[7] = 9
    b2 = make_batch([(b.pos, spec, b.cell[0])], 5)
    GMNN, DeviceSystem = _gm()
    m = GMNN(d, p)
    m.build_neighbors(DeviceSystem(b2), check=False)
    assert m.read_status() == _lib.GM_ERR_SPECIES


# ------------------------------------------------------------------ energies and forces

def _ef_parity(batch, desc, params, precision="fp32", virial=True):
    m, sysd, nl = _nl_pair(batch, desc, params)
    if precision != "fp32":
        m = _model(desc, params, precision)
    E, F, W = m.energy_forces(sysd, nl, virial=virial)
    m.check_status()
    ref = oracle.energy_forces(batch, desc, params, oracle.neighbors(batch, desc["r_cut"]))
    tol = TOL[precision]
    e = energy_error(E.cpu().numpy(), ref, batch)
    f_rms, f_max = force_error(F.cpu().numpy().astype(np.float64), ref)
    assert e <= tol, e
    assert f_rms <= tol, f_rms
    assert f_max <= ELEMENT_FACTOR * tol, f_max
    if virial:
        assert virial_error(W.cpu().numpy(), ref) <= tol
    return e, f_rms


@pytest.mark.parametrize("act", ["tanh", "silu"])
def test_energy_forces_config1(act):
    b, d, p = synth.config(1, activation=act)
    _ef_parity(b, d, p)


def test_energy_forces_ragged_li3po4_batch(li_small):
    b, d, p = li_small
    _ef_parity(b, d, p)


def test_energy_forces_config2_h512():
    b, d, p = synth.config(2)
    _ef_parity(b, d, p)


def test_energy_forces_emim_batch_with_empty_structure():
    b4, d, p = synth.config(4)
    b = subset(b4, [0, 3, 5])
    empty = (np.zeros((0, 3)), np.zeros(0, np.int32), 12.0 * np.eye(3))
    structs = [(b.pos[b.atom_ptr[k]:b.atom_ptr[k + 1]], b.species[b.atom_ptr[k]:b.atom_ptr[k + 1]], b.cell[k])
               for k in range(b.n_structures)]
    b = make_batch(structs[:1] + [empty] + structs[1:], 5)
    _ef_parity(b, d, p)


@pytest.mark.parametrize("cfg,act", [(1, "tanh"), (1, "silu"), (2, "silu")])
def test_energy_forces_mixed_precision(cfg, act):
    """BF16 network on tcgen05 tensor cores (FP32 accumulation), everything else FP32."""
    b, d, p = synth.config(cfg, activation=act)
    _ef_parity(b, d, p, precision="mixed")


@pytest.mark.parametrize("mask", [14, 15])
def test_energy_forces_mixed_split_masks(mask):
    """Other choices of the GEMMs that run the hi/lo split passes (the lo halves of the
    features and activations are written only where a split GEMM reads them)."""
    b, d, p = synth.config(1)
    m, sysd, nl = _nl_pair(b, d, p)
    mm = _model(d, p, "mixed")
    mm.set_tuning(split_mask=mask, f16_backward=0)     # the BF16 backward GEMMs the mask splits
    E, F, _ = mm.energy_forces(sysd, nl)
    mm.check_status()
    ref = oracle.energy_forces(b, d, p, oracle.neighbors(b, d["r_cut"]))
    e = energy_error(E.cpu().numpy(), ref, b)
    f_rms, f_max = force_error(F.cpu().numpy().astype(np.float64), ref)
    tol = 2e-4 if mask == 15 else TOL["mixed"]       # all four GEMMs split: close to FP32
    assert e <= tol and f_rms <= tol and f_max <= ELEMENT_FACTOR * tol, (e, f_rms, f_max)


@pytest.mark.parametrize("f16", [0, 1])
@pytest.mark.parametrize("cfg", [1, 2])
def test_energy_forces_mixed_backward_operand_formats(cfg, f16):
    """The two backward network GEMMs on FP16 operands in one pass (the default) or on BF16
    hi/lo pairs in three passes: both within the mixed tolerance of the oracle."""
    b, d, p = synth.config(cfg)
    m, sysd, nl = _nl_pair(b, d, p)
    mm = _model(d, p, "mixed")
    mm.set_tuning(f16_backward=f16)
    E, F, W = mm.energy_forces(sysd, nl, virial=True)
    mm.check_status()
    ref = oracle.energy_forces(b, d, p, oracle.neighbors(b, d["r_cut"]))
    tol = TOL["mixed"]
    e = energy_error(E.cpu().numpy(), ref, b)
    f_rms, f_max = force_error(F.cpu().numpy().astype(np.float64), ref)
    assert e <= tol and f_rms <= tol and f_max <= ELEMENT_FACTOR * tol, (e, f_rms, f_max)
    assert virial_error(W.cpu().numpy(), ref) <= tol


@pytest.mark.parametrize("act", ["tanh", "silu"])
@pytest.mark.parametrize("case", ["config1", "config2", "li_small"])
def test_fused_network_kernel_matches_oracle_and_the_four_gemms(case, act, li_small):
    """The mixed path's network as one tcgen05 kernel per 128-atom tile (widths 128, 512 and
    256 in these cases), forced on: within the mixed tolerance of the oracle, with virials,
    and within the same tolerance (RMS) of the four separate GEMMs, from which it differs by
    FP32 summation order and the FP16 rounding of phi'(z1) it keeps between its layers."""
    if case == "li_small":
        b, d, p = li_small
        d = dict(d, activation=act)
    else:
        b, d, p = synth.config(1 if case == "config1" else 2, activation=act)
    _, sysd, nl = _nl_pair(b, d, p)
    ref = oracle.energy_forces(b, d, p, oracle.neighbors(b, d["r_cut"]))
    outs = []
    for fused in (1, 0):
        mm = _model(d, p, "mixed")
        mm.set_tuning(fused_mlp=fused)
        E, F, W = mm.energy_forces(sysd, nl, virial=True)
        mm.check_status()
        _check_against(ref, b, E, F, W, TOL["mixed"])
        outs.append(F.cpu().numpy())
    rms = np.sqrt((ref["F"] ** 2).mean())
    assert np.sqrt(((outs[0] - outs[1]) ** 2).mean()) <= TOL["mixed"] * rms


@pytest.mark.parametrize("case,ctas", [("config2", 1), ("config2", 5), ("li_small", 7), ("emim8", 3)])
def test_persistent_fused_network_kernel_several_tiles_per_cta(case, ctas, li_small):
    """The one-CTA-per-tile network kernel is persistent: with fewer CTAs than tiles each CTA
    runs its tiles one after another (the next tile's G loading while the last epilogue runs,
    every barrier one phase per tile, the layers' MMAs and epilogue halves overlapping).
    Forced to 1-7 CTAs (widths 512, 256 and 128; 12-50 tiles): within the mixed tolerance of
    the oracle, and the same energies bit for bit as one CTA per SM (a tile's arithmetic does
    not depend on the CTA that runs it), forces up to the order of their atomic sums."""
    if case == "li_small":
        b, d, p = li_small
    elif case == "emim8":
        b, d, p = synth.config(4)
        b = subset(b, range(8))
    else:
        b, d, p = synth.config(2)
    _, sysd, nl = _nl_pair(b, d, p)
    ref = _oracle_ref(case, b, d, p)
    outs = []
    for c in (ctas, 0):
        mm = _model(d, p, "mixed")
        mm.set_tuning(fused_mlp=1, mlp_cluster=1, mlp_ctas=c)
        E, F, W = mm.energy_forces(sysd, nl, virial=True)
        mm.check_status()
        _check_against(ref, b, E, F, W, TOL["mixed"])
        outs.append((E.cpu().numpy(), F.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.abs(outs[0][1] - outs[1][1]).max() <= 1e-5 * np.abs(outs[1][1]).max()


@pytest.mark.parametrize("bn", [64, 128, 256])
def test_mixed_gemm_blocks_per_sm_give_identical_results(bn):
    """One or two tensor-core GEMM blocks per SM (a full or a halved operand ring) compute each
    output tile the same way: energies agree bit for bit, forces up to the order of their FP32
    atomic sums, and both are within the mixed tolerance of the oracle."""
    b, d, p = synth.config(2)
    _, sysd, nl = _nl_pair(b, d, p)
    ref = oracle.energy_forces(b, d, p, oracle.neighbors(b, d["r_cut"]))
    outs = []
    for cps in (1, 2):
        mm = _model(d, p, "mixed")
        mm.set_tuning(gemm_bn=bn, gemm_cps=cps)
        E, F, _ = mm.energy_forces(sysd, nl)
        mm.check_status()
        outs.append((E.cpu().numpy(), F.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.abs(outs[0][1] - outs[1][1]).max() <= 1e-5 * np.abs(outs[0][1]).max()
    e = energy_error(outs[1][0], ref, b)
    f_rms, f_max = force_error(outs[1][1].astype(np.float64), ref)
    tol = TOL["mixed"]
    assert e <= tol and f_rms <= tol and f_max <= ELEMENT_FACTOR * tol, (e, f_rms, f_max)


def test_energy_forces_mixed_ragged_li3po4_batch(li_small):
    b, d, p = li_small
    _ef_parity(b, d, p, precision="mixed")


def test_autotuned_batched_model_matches_oracle(li_small):
    """The autotuner's choice (over a reduced knob space) keeps energies and forces within the
    parity tolerance of the oracle."""
    from paper_2505_22168_b300 import autotune, NeighborList
    GMNN, DeviceSystem = _gm()
    b, d, p = li_small
    for precision in ("fp32", "mixed"):
        m = GMNN(d, p, precision=precision)
        sysd = DeviceSystem(b)
        nl0 = m.build_neighbors(sysd)
        nl = NeighborList(b.n_atoms, nl0.capacity, m.device)
        out = (torch.empty(b.n_structures, dtype=torch.float64, device=m.device),
               torch.empty(b.n_atoms, 3, dtype=torch.float32, device=m.device), None)
        space = {"nl_items": (0, 1, 2), "pair_tpa": (0, 8, 32), "forces_tpa": (0, 16), "gemm_bn": (0, 128)}
        r = autotune.tune(m, sysd, nl, out, reps=3, space=space)
        assert set(r["settings"]) <= set(space)
        m.step(sysd, nl, out)
        m.check_status()
        ref = oracle.energy_forces(b, d, p, oracle.neighbors(b, d["r_cut"]))
        tol = TOL[precision]
        assert energy_error(out[0].cpu().numpy(), ref, b) <= tol
        rms, worst = force_error(out[1].cpu().numpy().astype(np.float64), ref)
        assert rms <= tol and worst <= ELEMENT_FACTOR * tol


def test_descriptors_match_oracle():
    b, d, p = synth.config(1)
    m, sysd, nl = _nl_pair(b, d, p)
    psi, G = m.descriptors(sysd, nl)
    m.check_status()
    ref = oracle.energy_forces(b, d, p, oracle.neighbors(b, d["r_cut"]), psi=True, features=True)
    scale_psi = np.abs(ref["psi"]).max()
    assert np.abs(psi.cpu().numpy() - ref["psi"]).max() <= 1e-5 * scale_psi
    for lo, hi in ((0, 5), (5, 20), (20, 35), (35, 50), (50, 85), (85, 160), (160, 235), (235, 360)):
        g, r = G.cpu().numpy()[:, lo:hi], ref["G"][:, lo:hi]
        assert np.abs(g - r).max() <= 1e-5 * np.abs(r).max(), (lo, hi)


def test_energy_forces_deterministic_energy():
    b, d, p = synth.config(1)
    m, sysd, nl = _nl_pair(b, d, p)
    E1, _, _ = m.energy_forces(sysd, nl)
    E2, _, _ = m.energy_forces(sysd, nl)
    assert float(E1.item()) == float(E2.item())


def test_batched_energies_and_virials_are_deterministic(li_small):
    """Structure sums are exact integer sums (fixed point): repeated steps on a ragged batch
    give identical energies and virials although the order of the block atomics varies."""
    b, d, p = li_small
    m, sysd, nl = _nl_pair(b, d, p)
    runs = [m.energy_forces(sysd, nl, virial=True) for _ in range(3)]
    for E, _, W in runs[1:]:
        assert torch.equal(E, runs[0][0]) and torch.equal(W, runs[0][2])


def _with_empty_structure():
    b4, d, p = synth.config(4)
    b = subset(b4, [0, 3, 5])
    empty = (np.zeros((0, 3)), np.zeros(0, np.int32), 12.0 * np.eye(3))
    structs = [(b.pos[b.atom_ptr[k]:b.atom_ptr[k + 1]], b.species[b.atom_ptr[k]:b.atom_ptr[k + 1]], b.cell[k])
               for k in range(b.n_structures)]
    return make_batch(structs[:1] + [empty] + structs[1:], 5), d, p


@pytest.mark.parametrize("which", ["emim1536", "li3po4_batch", "with_empty"])
def test_mixed_energies_summed_in_gemm_equal_reduction_kernel(which, li_small):
    """Without the virial the mixed path sums the structure energies inside its first
    backward GEMM; with it, the reduction kernel does.  Both add the same per-atom FP32
    energies as exact fixed-point integers, so the energies agree bit for bit, and they are
    within the mixed tolerance of the oracle.  (The forces take neighbour contributions by
    float atomics, so they agree to rounding.)"""
    if which == "emim1536":
        b, d, p = synth.config(2)
    elif which == "li3po4_batch":
        b, d, p = li_small
    else:
        b, d, p = _with_empty_structure()
    _ef_parity(b, d, p, precision="mixed", virial=False)
    _, sysd, nl = _nl_pair(b, d, p)
    mm = _model(d, p, "mixed")
    E0, F0, _ = mm.energy_forces(sysd, nl, virial=False)
    E1, F1, _ = mm.energy_forces(sysd, nl, virial=True)
    mm.check_status()
    assert np.array_equal(E0.cpu().numpy(), E1.cpu().numpy(), equal_nan=True)
    f0, f1 = F0.cpu().numpy(), F1.cpu().numpy()    # float atomics: summation order varies
    assert np.abs(f0 - f1).max() <= 1e-5 * max(np.abs(f1).max(), 1e-30)


def test_diverged_energy_comes_out_nan_mixed_without_virial():
    """The NaN rule of the structure sums holds where the mixed path sums the energies
    inside its GEMM (no virial)."""
    b1, d, p = synth.config(1)
    spec1 = np.ones_like(b1.species)
    b = make_batch([(b1.pos, b1.species, b1.cell[0]), (b1.pos, spec1, b1.cell[0]),
                    (b1.pos, b1.species, b1.cell[0])], d["n_species"])
    p = dict(p)
    p["mu"] = np.array(p["mu"], dtype=np.float64).copy()
    p["mu"][0] = 2e9
    _, sysd, nl = _nl_pair(b, d, p)
    mm = _model(d, p, "mixed")
    E, _, _ = mm.energy_forces(sysd, nl, virial=False)
    mm.check_status()
    has0 = [bool((b.species[b.atom_ptr[k]:b.atom_ptr[k + 1]] == 0).any()) for k in range(b.n_structures)]
    E = E.cpu().numpy()
    assert any(has0) and not all(has0)
    for k in range(b.n_structures):
        assert np.isnan(E[k]) == has0[k]


def test_diverged_energy_comes_out_nan():
    """A per-atom energy beyond the fixed-point range (here an energy shift of 2e9 for one
    species) makes the structures holding that species NaN instead of wrapping around."""
    b1, d, p = synth.config(1)
    spec1 = np.ones_like(b1.species)                     # a copy of the box without species 0
    b = make_batch([(b1.pos, b1.species, b1.cell[0]), (b1.pos, spec1, b1.cell[0]),
                    (b1.pos, b1.species, b1.cell[0])], d["n_species"])
    p = dict(p)
    p["mu"] = np.array(p["mu"], dtype=np.float64).copy()
    p["mu"][0] = 2e9
    m, sysd, nl = _nl_pair(b, d, p)
    E, _, W = m.energy_forces(sysd, nl, virial=True)
    m.check_status()
    has0 = [bool((b.species[b.atom_ptr[k]:b.atom_ptr[k + 1]] == 0).any()) for k in range(b.n_structures)]
    E = E.cpu().numpy()
    assert any(has0)
    for k in range(b.n_structures):
        assert np.isnan(E[k]) == has0[k]


# ------------------------------------------------------------------ full size

def test_full_size_li3po4_sampled_rows_and_properties():
    """131,072 atoms (launch configuration of the benchmark): the neighbour rows and the
    descriptors of 48 sampled atoms equal the oracle's; every pair has its mirror
    (j, i, -n); the net force vanishes."""
    b, d, p = synth.config(5)
    m, sysd, nl = _nl_pair(b, d, p)
    E, F, _ = m.energy_forces(sysd, nl)
    m.check_status()
    psi, G = m.descriptors(sysd, nl)
    m.check_status()
    rows = np.sort(np.random.default_rng(9).choice(b.n_atoms, 48, replace=False))
    t = nl.triples()
    onl = oracle.neighbor_rows(b, d["r_cut"], rows)
    assert np.array_equal(t[np.isin(t[:, 0], rows)], onl.triples())
    opsi, oG = oracle.descriptors(b, d, p, onl, rows)
    assert np.abs(psi.cpu().numpy()[rows] - opsi).max() <= 1e-5 * np.abs(opsi).max()
    assert np.abs(G.cpu().numpy()[rows] - oG).max() <= 1e-5 * np.abs(oG).max()
    mirror = np.column_stack([t[:, 1], t[:, 0], -t[:, 2], -t[:, 3], -t[:, 4]])
    mirror = mirror[np.lexsort(mirror.T[::-1])]
    assert np.array_equal(t, mirror)
    Fn = F.cpu().numpy().astype(np.float64)
    assert np.abs(Fn.sum(0)).max() <= 1e-4 * np.sqrt((Fn ** 2).mean()) * np.sqrt(b.n_atoms)
    assert np.isfinite(E.cpu().numpy()).all()


# ------------------------------------------------------------------ lanes per atom

_REFS = {}


def _oracle_ref(key, batch, desc, params):
    """Oracle energies, forces and virials, computed once per system of this module."""
    if key not in _REFS:
        _REFS[key] = oracle.energy_forces(batch, desc, params, oracle.neighbors(batch, desc["r_cut"]))
    return _REFS[key]


def _check_against(ref, batch, E, F, W, tol):
    e = energy_error(E.cpu().numpy(), ref, batch)
    f_rms, f_max = force_error(F.cpu().numpy().astype(np.float64), ref)
    assert e <= tol and f_rms <= tol and f_max <= ELEMENT_FACTOR * tol, (e, f_rms, f_max)
    if W is not None:
        v = virial_error(W.cpu().numpy(), ref)
        assert v <= tol, v
    return e, f_rms, f_max


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
@pytest.mark.parametrize("tpa", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("case", ["config1", "li_small"])
def test_energy_forces_every_pair_lane_count(case, tpa, precision, li_small):
    """Every lanes-per-atom shape of the pair kernels (moments: 1 lane, 2 and 4 lanes with the
    component split over lane pairs, 8-32 with the reduce-scatter; forces: 1 and 2 lanes
    without the shared-memory dE/dPsi rows, 4-32 with them) against the oracle, with the
    virial, on the 96-atom box and on 24 Li3PO4 boxes (several with multiple images)."""
    b, d, p = synth.config(1) if case == "config1" else li_small
    ref = _oracle_ref(case, b, d, p)
    GMNN, DeviceSystem = _gm()
    m = GMNN(d, p, precision=precision)
    m.set_tuning(pair_tpa=tpa)
    from paper_2505_22168_b300 import _lib
    assert _lib.gm_model_pair_lanes(m.handle, b.n_atoms) == tpa
    assert _lib.gm_model_force_lanes(m.handle, b.n_atoms) == tpa
    sysd = DeviceSystem(b)
    nl = m.build_neighbors(sysd)
    E, F, W = m.energy_forces(sysd, nl, virial=True)
    m.check_status()
    _check_against(ref, b, E, F, W, TOL[precision])


def _li_boxes(n_boxes):
    """n_boxes Li3PO4-like crystals of 512 atoms each (17.2 A, single image at r_cut 6) with
    the 131,072-atom workload's model (r_cut 6, 2x512): the library's own lanes-per-atom
    choice depends on the total atom count only."""
    from synth.systems import li3po4_crystal
    _, d, p = synth.config(5)
    b = make_batch([li3po4_crystal(64, 7100 + k, sigma=0.1) for k in range(n_boxes)], 3)
    return b, d, p


@pytest.mark.parametrize("n_boxes,lanes,force_lanes", [(16, 32, 8), (32, 4, 8), (64, 2, 8), (96, 2, 4)])
def test_library_lane_choice_by_size_matches_oracle(n_boxes, lanes, force_lanes):
    """8,192, 16,384, 32,768 and 49,152 atoms: the pair-kernel shapes the library picks by size
    for mid-size and large systems (moments 32 lanes per atom with the reduce-scatter kernel,
    then 4, 2 and 2 with the component-split kernel; forces 8, then 4 from 49,152 atoms, as for
    the 131,072-atom crystal and the batched Li3PO4 workload), with no forced knob, against the
    full oracle for both precisions, energies, forces and virials."""
    b, d, p = _li_boxes(n_boxes)
    ref = _oracle_ref(("li_boxes", n_boxes), b, d, p)
    GMNN, DeviceSystem = _gm()
    from paper_2505_22168_b300 import _lib
    for precision in ("fp32", "mixed"):
        m = GMNN(d, p, precision=precision)
        assert _lib.gm_model_pair_lanes(m.handle, b.n_atoms) == lanes
        assert _lib.gm_model_force_lanes(m.handle, b.n_atoms) == force_lanes
        sysd = DeviceSystem(b)
        nl = m.build_neighbors(sysd)
        E, F, W = m.energy_forces(sysd, nl, virial=True)
        m.check_status()
        _check_against(ref, b, E, F, W, TOL[precision])
        E2, F2, _ = m.energy_forces(sysd, nl, virial=False)       # the step the benchmark times
        m.check_status()
        _check_against(ref, b, E2, F2, None, TOL[precision])


def test_full_size_li3po4_sampled_forces_match_oracle():
    """131,072 atoms in the benchmark's launch configuration (moments two lanes per atom with
    the component-split kernel, forces four, the fused network kernel): the forces
    and the atomic energies of 12 sampled atoms equal an exact oracle evaluation of those atoms
    (their neighbours' complete environments are evaluated; nothing is truncated), for both
    precisions."""
    b, d, p = synth.config(5)
    rows = np.sort(np.random.default_rng(21).choice(b.n_atoms, 12, replace=False))
    ref = oracle.sampled_forces(b, d, p, rows)
    GMNN, DeviceSystem = _gm()
    from paper_2505_22168_b300 import _lib
    for precision in ("fp32", "mixed"):
        m = GMNN(d, p, precision=precision)
        assert _lib.gm_model_pair_lanes(m.handle, b.n_atoms) == 2
        assert _lib.gm_model_force_lanes(m.handle, b.n_atoms) == 4
        sysd = DeviceSystem(b)
        nl = m.build_neighbors(sysd)
        _, F, _ = m.energy_forces(sysd, nl, virial=False)
        m.check_status()
        Fs = F.cpu().numpy().astype(np.float64)[ref["rows"]]
        rms = np.sqrt((ref["F"] ** 2).mean())
        tol = TOL[precision]
        f_rms = np.sqrt(((Fs - ref["F"]) ** 2).mean()) / rms
        f_max = np.abs(Fs - ref["F"]).max() / rms
        assert f_rms <= tol and f_max <= ELEMENT_FACTOR * tol, (precision, f_rms, f_max)
