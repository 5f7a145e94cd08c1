"""GPU molecular dynamics (gm_md_init / gm_md_run) against the FP64 MD reference (oracle.md),
through the C ABI: velocity Verlet and the Nose-Hoover chain step by step, the skin list
rebuilt on the device only when an atom has moved more than skin/2, CUDA-graph replay of
the inner steps, and batches of structures with their own chains."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from oracle import md as omd
from synth.params import maxwell_boltzmann
from synth.systems import li3po4_crystal, make_batch, species_masses
from tests.parity import TOL, energy_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_22168_b300 import build
    build.build()


def _system(units=(24,), seed=777):
    _, d, p = synth.config(3)
    b = make_batch([li3po4_crystal(u, seed + k, sigma=0.05) for k, u in enumerate(units)], 3)
    masses = species_masses("li3po4")
    vel = maxwell_boltzmann(masses[b.species], b.atom_ptr, 600.0, seed)
    return b, d, p, masses, vel


def _gpu_md(b, d, p, masses, vel, params, n_steps, precision="fp32", chunks=1, graph=False, tune=None):
    from paper_2505_22168_b300 import GMNN, DeviceSystem, MDState
    m = GMNN(d, p, precision=precision)
    if tune:
        m.set_tuning(**tune)
    sysd = DeviceSystem(b)
    nl = m.md_neighbor_list(sysd, params)
    st = MDState(sysd, masses, vel)
    m.md_init(sysd, nl, params, st)
    per = n_steps // chunks
    if graph:
        g = m.capture_md(sysd, nl, params, st, per)
        for _ in range(chunks):
            g.replay()
    else:
        for _ in range(chunks):
            m.md_run(sysd, nl, params, st, per)
    m.check_status()
    return m, sysd, nl, st


def _oracle_md(b, d, p, masses, vel, params, n_steps):
    nvt = None
    if params.ensemble == "nvt":
        nvt = {"temperature": params.temperature, "tau": params.tau, "chain_length": params.chain_length,
               "chain_steps": params.chain_steps, "sy_steps": params.sy_steps}
    return omd.integrate(b.pos, vel, masses[b.species], b.atom_ptr, omd.gmnn_force_fn(b, d, p), params.dt, n_steps,
                         nvt=nvt)


# bounds after the run: the FP32 path's forces are within ~1e-6 of the FP64 ones, the mixed
# path's within ~1e-3; over tens of steps that moves atoms by ~1e-9 and ~1e-6 A.  The
# thermostat chain itself runs in FP32 on both paths (its thermostat positions in FP64), so
# its state carries FP32 rounding, amplified by a strongly coupled chain (tau = 10 steps).
BOUNDS = {"fp32": {"pos": 1e-6, "vel": 1e-7, "ke": 1e-6, "chain": 1e-4},
          "mixed": {"pos": 1e-4, "vel": 1e-5, "ke": 1e-4, "chain": 1e-3}}


def _compare(st, ref, b, masses, params, precision, n_steps):
    pos, vel, E, F, chains = ref
    bd = BOUNDS[precision]
    assert np.abs(st.pos.cpu().numpy() - pos).max() <= bd["pos"]
    assert np.abs(st.vel.cpu().numpy() - vel).max() <= bd["vel"]
    ke_ref = omd.kinetic(vel, masses[b.species], b.atom_ptr)
    assert np.abs(st.kinetic.cpu().numpy() - ke_ref).max() <= bd["ke"] * np.abs(ke_ref).max()
    assert energy_error(st.energy.cpu().numpy(), {"E": E, "E_atom": np.full(b.n_atoms, np.abs(E).max() / b.n_atoms)},
                        b) <= TOL[precision]
    F_got = st.forces.cpu().numpy().astype(np.float64)
    rms = np.sqrt((F ** 2).mean())
    assert np.sqrt(((F_got - F) ** 2).mean()) / rms <= TOL[precision] * 10
    if chains is not None:
        ch = st.chain.cpu().numpy()
        for k, c in enumerate(chains):
            M = c.M
            scale = max(np.abs(c.v).max(), 1e-12)
            assert np.abs(ch[k, 1, :M] - c.v).max() <= bd["chain"] * scale
            assert np.abs(ch[k, 0, :M] - c.xi).max() <= bd["chain"] * max(np.abs(c.xi).max(), 1e-12)


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
@pytest.mark.parametrize("ensemble", ["nve", "nvt"])
def test_md_matches_oracle_with_skin_rebuilds(ensemble, precision):
    """120 steps of 0.5 fs at 600 K on a 192-atom Li3PO4-like box with a 0.2 A skin (the list is
    rebuilt every few tens of steps): positions, velocities, energies, forces and chain state
    follow the FP64 reference that recomputes its neighbours from scratch every step."""
    from paper_2505_22168_b300 import MDParams
    b, d, p, masses, vel = _system()
    params = MDParams(dt=0.5, skin=0.2, temperature=600.0, tau=5.0, ensemble=ensemble)
    n = 120
    _, _, _, st = _gpu_md(b, d, p, masses, vel, params, n, precision)
    builds = int(st.n_builds.item())
    assert 3 <= builds < n // 4, builds                   # the list was reused between rebuilds
    ref = _oracle_md(b, d, p, masses, vel, params, n)
    _compare(st, ref, b, masses, params, precision, n)


@pytest.mark.parametrize("cs", [1, 2, 4])
def test_md_with_the_fused_network_kernels(cs):
    """The same NVT run on the mixed path with the network as one kernel per tile (cs 1) or a
    cluster of 2 or 4 CTAs per tile (the forms the library picks for mid-size and large MD
    systems; the 192-atom box would take the four GEMM launches): the same bounds."""
    from paper_2505_22168_b300 import MDParams
    b, d, p, masses, vel = _system()
    params = MDParams(dt=0.5, skin=0.2, temperature=600.0, tau=5.0, ensemble="nvt")
    n = 120
    _, _, _, st = _gpu_md(b, d, p, masses, vel, params, n, "mixed", graph=True,
                          tune=dict(fused_mlp=1, mlp_cluster=cs))
    ref = _oracle_md(b, d, p, masses, vel, params, n)
    _compare(st, ref, b, masses, params, "mixed", n)


def test_skin_list_holds_every_pair_within_the_cutoff():
    """After a run, the list (built some steps ago at r_cut + skin) restricted to pairs within
    r_cut at the current positions is exactly the brute-force r_cut list of those positions."""
    from paper_2505_22168_b300 import MDParams
    b, d, p, masses, vel = _system()
    params = MDParams(dt=0.5, skin=0.5, ensemble="nve")
    _, sysd, nl, st = _gpu_md(b, d, p, masses, vel, params, 40)
    pos = st.pos.cpu().numpy()
    t = nl.triples()
    L = b.cell[0].diagonal()
    dvec = pos[t[:, 1]] - pos[t[:, 0]] + t[:, 2:5] * L
    r2 = (dvec[:, 0] * dvec[:, 0] + dvec[:, 1] * dvec[:, 1]) + dvec[:, 2] * dvec[:, 2]
    inside = t[r2 < d["r_cut"] ** 2]
    want = oracle.neighbors(dataclasses.replace(b, pos=pos), d["r_cut"]).triples()
    assert np.array_equal(inside, want)
    assert len(t) > len(want)                              # the skin pairs are there too


def test_md_graph_replay_matches_stream_launches():
    """Three replays of a captured 20-step run equal three 20-step runs launched on the stream."""
    from paper_2505_22168_b300 import MDParams
    b, d, p, masses, vel = _system()
    params = MDParams(dt=0.5, skin=0.3, ensemble="nvt", tau=5.0)
    _, _, _, a = _gpu_md(b, d, p, masses, vel, params, 60, chunks=3)
    _, _, _, g = _gpu_md(b, d, p, masses, vel, params, 60, chunks=3, graph=True)
    # the force kernel adds neighbour contributions with float atomics, so two runs differ in
    # the last bits of the forces; after 60 steps that is ~1e-9 A
    assert np.abs(a.pos.cpu().numpy() - g.pos.cpu().numpy()).max() <= 1e-7
    assert np.abs(a.vel.cpu().numpy() - g.vel.cpu().numpy()).max() <= 1e-8
    assert int(a.n_builds.item()) == int(g.n_builds.item())


def test_md_batch_of_structures_with_their_own_chains():
    """Three boxes of 64, 192 and 512 atoms integrated together: each has its own chain and
    follows the reference."""
    from paper_2505_22168_b300 import MDParams
    b, d, p, masses, vel = _system(units=(8, 24, 64), seed=900)
    params = MDParams(dt=0.5, skin=0.3, ensemble="nvt", tau=5.0)
    _, _, _, st = _gpu_md(b, d, p, masses, vel, params, 40)
    ref = _oracle_md(b, d, p, masses, vel, params, 40)
    _compare(st, ref, b, masses, params, "fp32", 40)


def test_md_capacity_overflow_is_reported_and_freezes_the_state():
    from paper_2505_22168_b300 import GMNN, DeviceSystem, MDParams, MDState, NeighborList, _lib
    b, d, p, masses, vel = _system()
    params = MDParams(dt=0.5, skin=0.5, ensemble="nve")
    m = GMNN(d, p)
    sysd = DeviceSystem(b)
    nl = NeighborList(b.n_atoms, 1000, m.device)
    st = MDState(sysd, masses, vel)
    m.md_init(sysd, nl, params, st)
    m.md_run(sysd, nl, params, st, 5)
    assert m.read_status() == _lib.GM_ERR_CAPACITY
    assert np.array_equal(st.pos.cpu().numpy(), b.pos)          # nothing moved
    assert np.isfinite(st.vel.cpu().numpy()).all()
