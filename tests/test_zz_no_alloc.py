"""gm_build_neighbors_noalloc: the neighbour build for callers that cannot give the
library device memory (a host program whose allocator owns all of it, or a step loop that
must not call cudaMalloc).  It must produce exactly the neighbour list of
gm_build_neighbors, call after call, although every call reuses the same fixed scratch
array inside the library.  Integer output, so the comparison is bit for bit.

This file is collected last on purpose, and it passes both alone in a fresh process and
after the other tests (its first call may be the one that looks up the scratch address).
"""
import numpy as np
import pytest

import synth
from tests.parity import subset

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_22168_b300 import build
    build.build()


def _lists(model, sysd, capacity):
    from paper_2505_22168_b300 import NeighborList
    return NeighborList(sysd.n_atoms, capacity, model.device), NeighborList(sysd.n_atoms, capacity, model.device)


def _host(nl):
    P = int(nl.n_pairs.item())
    return (nl.row_ptr.cpu().numpy(), nl.col[:P].cpu().numpy(), nl.shift[:P].cpu().numpy(), P)


def _compare_once(batch, desc, params, **tuning):
    from paper_2505_22168_b300 import GMNN, DeviceSystem, _lib
    from paper_2505_22168_b300.gmnn import _ptr, _stream
    model = GMNN(desc, params)
    model.set_tuning(**tuning)
    sysd = DeviceSystem(batch)
    cap = model.estimate_capacity(sysd)
    ref, got = _lists(model, sysd, cap)
    # existing entry point, with a caller-provided workspace
    ws, wsb = model.workspace(_lib.GM_OP_NEIGHBORS, sysd, cap)
    model.clear_status()
    _lib.gm_build_neighbors(model.handle, sysd.c_struct(), ref.c_struct(), ws, wsb, _ptr(model.status), _stream())
    assert model.read_status() == _lib.GM_OK
    # the variant without workspace
    model.clear_status()
    _lib.gm_build_neighbors_noalloc(model.handle, sysd.c_struct(), got.c_struct(), _ptr(model.status), _stream())
    assert model.read_status() == _lib.GM_OK
    a, b = _host(ref), _host(got)
    assert a[3] == b[3] and a[3] > 0
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)


def test_noalloc_matches_workspace_build_on_two_calls_in_a_row():
    b1, d1, p1 = synth.config(1)
    b3, d3, p3 = synth.config(3)
    _compare_once(b1, d1, p1)                          # first call (may set up the scratch address)
    _compare_once(subset(b3, range(40)), d3, p3)       # second call: other system, stale scratch
    _compare_once(b1, d1, p1)                          # and back


def test_noalloc_two_pass_search_matches_workspace_build():
    """Systems whose search slab does not fit beside the minimum workspace in the fixed
    scratch take the two-pass search (count, then fill): a 32,768-atom Li3PO4-like crystal
    at r_cut 6 (minimum workspace ~3 MB, slab ~17 MB), and the 96-atom box with the
    two-pass search forced on both entry points."""
    from synth.systems import li3po4_crystal, make_batch
    b5, d5, p5 = synth.config(5)
    big = make_batch([li3po4_crystal(4096, 2024, sigma=0.1)], b5.n_species)
    _compare_once(big, d5, p5)
    b1, d1, p1 = synth.config(1)
    _compare_once(b1, d1, p1, nl_two_pass=1)


def test_noalloc_rejects_a_misaligned_position_pointer():
    """The same host-side argument checks as gm_build_neighbors: a position pointer that is
    not 8-byte aligned returns GM_ERR_ARG before anything is launched."""
    from paper_2505_22168_b300 import GMNN, DeviceSystem, NeighborList, _lib
    from paper_2505_22168_b300.gmnn import _ptr, _stream
    b, d, p = synth.config(1)
    model = GMNN(d, p)
    sysd = DeviceSystem(b)
    sysc = sysd.c_struct()
    sysc.pos = _ptr(sysd.pos) + 4
    nl = NeighborList(b.n_atoms, 16, model.device)
    with pytest.raises(_lib.GmError) as e:
        _lib.gm_build_neighbors_noalloc(model.handle, sysc, nl.c_struct(), _ptr(model.status), _stream())
    assert e.value.code == _lib.GM_ERR_ARG
    torch.cuda.synchronize()
    assert model.read_status() == _lib.GM_OK


def test_noalloc_rejects_systems_beyond_its_fixed_scratch():
    from paper_2505_22168_b300 import GMNN, NeighborList, _lib
    from paper_2505_22168_b300.gmnn import _ptr, _stream
    b, d, p = synth.config(1)
    model = GMNN(d, p)
    n_big = 200_000
    dummy_i = torch.zeros(4, dtype=torch.int32, device=model.device)
    dummy_d = torch.zeros(16, dtype=torch.float64, device=model.device)
    dummy_u = torch.ones(3, dtype=torch.uint8, device=model.device)
    sysc = _lib.GmSystem(1, n_big, _ptr(dummy_i), _ptr(dummy_d), _ptr(dummy_i), _ptr(dummy_d), _ptr(dummy_u))
    nl = NeighborList(4, 16, model.device)
    with pytest.raises(_lib.GmError) as e:
        _lib.gm_build_neighbors_noalloc(model.handle, sysc, nl.c_struct(), _ptr(model.status), _stream())
    assert e.value.code == _lib.GM_ERR_WORKSPACE
    assert "8 MiB" in str(e.value)
