"""Failure reporting of the bounded device waits, made to run out on purpose.

Every wait in the library's kernels is bounded (about one second): the grid barriers of the
cooperative neighbour build and the mbarrier waits of the tcgen05 GEMM and of the fused
network kernels.  A test-only knob (GM_TUNE_DEBUG_STALL) removes one participant -- block 0 of
the neighbour build never arrives at its barrier, or the GEMM's (the fused kernel's) producer
issues no loads -- so that the other waits expire with nothing asynchronous in flight.  The status word must read GM_ERR_TIMEOUT, the
call's later kernels skip their work, and the next call with the knob off returns the
oracle's results.  No GPU faults, traps or hangs: every waiting block returns.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.parity import ELEMENT_FACTOR, TOL, energy_error, force_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_22168_b300 import build
    build.build()


def test_grid_barrier_timeout_is_reported_and_the_next_build_is_clean():
    from paper_2505_22168_b300 import GMNN, DeviceSystem, _lib
    b, d, p = synth.config(2)
    m = GMNN(d, p)
    sysd = DeviceSystem(b)
    nl = m.build_neighbors(sysd)
    m.set_tuning(debug_stall=1)
    m.build_neighbors(sysd, nl, check=False)
    assert m.read_status() == _lib.GM_ERR_TIMEOUT
    m.set_tuning(debug_stall=0)
    nl = m.build_neighbors(sysd, nl)                      # same buffers and workspace
    assert m.read_status() == _lib.GM_OK
    assert np.array_equal(nl.triples(), oracle.neighbors(b, d["r_cut"]).triples())


def test_tcgen05_gemm_wait_timeout_is_reported_and_the_next_call_is_clean():
    from paper_2505_22168_b300 import GMNN, DeviceSystem, _lib
    b, d, p = synth.config(1)
    m = GMNN(d, p, precision="mixed")
    sysd = DeviceSystem(b)
    nl = m.build_neighbors(sysd)
    m.set_tuning(debug_stall=2)
    m.energy_forces(sysd, nl)
    assert m.read_status() == _lib.GM_ERR_TIMEOUT
    m.set_tuning(debug_stall=0)
    E, F, _ = m.energy_forces(sysd, nl)
    assert m.read_status() == _lib.GM_OK
    ref = oracle.energy_forces(b, d, p, oracle.neighbors(b, d["r_cut"]))
    tol = TOL["mixed"]
    f_rms, f_max = force_error(F.cpu().numpy().astype(np.float64), ref)
    assert energy_error(E.cpu().numpy(), ref, b) <= tol and f_rms <= tol and f_max <= ELEMENT_FACTOR * tol


@pytest.mark.parametrize("cs", [1, 4])
def test_fused_network_wait_timeout_is_reported_and_the_next_call_is_clean(cs):
    """The fused network kernel, one CTA per tile (cs 1) or a cluster of 4 per tile, with a
    producer that issues no loads: every CTA's waits run out (the cluster's CTAs still meet at
    their final barrier), GM_ERR_TIMEOUT is reported, and the next call is correct."""
    from paper_2505_22168_b300 import GMNN, DeviceSystem, _lib
    b, d, p = synth.config(2)
    m = GMNN(d, p, precision="mixed")
    sysd = DeviceSystem(b)
    nl = m.build_neighbors(sysd)
    m.set_tuning(fused_mlp=1, mlp_cluster=cs, debug_stall=2)
    m.energy_forces(sysd, nl)
    assert m.read_status() == _lib.GM_ERR_TIMEOUT
    m.set_tuning(debug_stall=0)
    E, F, _ = m.energy_forces(sysd, nl)
    assert m.read_status() == _lib.GM_OK
    ref = oracle.energy_forces(b, d, p, oracle.neighbors(b, d["r_cut"]))
    tol = TOL["mixed"]
    f_rms, f_max = force_error(F.cpu().numpy().astype(np.float64), ref)
    assert energy_error(E.cpu().numpy(), ref, b) <= tol and f_rms <= tol and f_max <= ELEMENT_FACTOR * tol
