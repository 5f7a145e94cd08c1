"""PyTorch-facing wrapper of libgm: device buffers, streams and an autograd Function.

PyTorch supplies device memory and the current CUDA stream; every computation runs in
libgm's kernels through the C ABI (``_lib``).  Nothing here computes model arithmetic.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import _lib as L

PARAM_ORDER = ("beta", "W1", "b1", "W2", "b2", "w3", "b3", "sigma", "mu")
ACT = {"tanh": L.GM_ACT_TANH, "silu": L.GM_ACT_SILU}
PREC = {"fp32": L.GM_PREC_FP32, "mixed": L.GM_PREC_MIXED}
BASIS = {"gaussian": L.GM_BASIS_GAUSSIAN, "bessel": L.GM_BASIS_BESSEL}


def pack_theta(params) -> np.ndarray:
    """Flat FP32 parameter vector in the order of include/gm.h."""
    return np.concatenate([np.asarray(params[k], np.float64).reshape(-1) for k in PARAM_ORDER]).astype(np.float32)


def unpack_theta(theta, n_species, n_hidden, n_radial=5, n_basis=7, n_ensemble=1):
    """Inverse of pack_theta: dict of named arrays (numpy)."""
    from synth.params import param_shapes  # shapes only
    th = np.asarray(theta)
    out, off = {}, 0
    for k, shp in param_shapes(n_species, n_hidden, n_radial, n_basis, n_ensemble=n_ensemble).items():
        n = int(np.prod(shp))
        out[k] = th[off:off + n].reshape(shp)
        off += n
    return out


def _ptr(t):
    return 0 if t is None else int(t.data_ptr())


def _stream():
    return int(torch.cuda.current_stream().cuda_stream)


class DeviceSystem:
    """A batch of periodic structures resident on the GPU (the gm_system of the C ABI)."""

    def __init__(self, batch, device="cuda"):
        dev = torch.device(device)
        self.n_structures = int(batch.n_structures)
        self.n_atoms = int(batch.n_atoms)
        self.atom_ptr = torch.as_tensor(np.asarray(batch.atom_ptr, np.int32), device=dev)
        self.pos = torch.as_tensor(np.asarray(batch.pos, np.float64), device=dev).contiguous()
        self.species = torch.as_tensor(np.asarray(batch.species, np.int32), device=dev)
        self.cell = torch.as_tensor(np.asarray(batch.cell, np.float64).reshape(-1, 9), device=dev).contiguous()
        self.pbc = torch.as_tensor(np.asarray(batch.pbc, np.uint8).reshape(-1, 3), device=dev).contiguous()
        self.host_counts = np.diff(np.asarray(batch.atom_ptr))
        self.host_cells = np.asarray(batch.cell, np.float64).reshape(-1, 3, 3)

    def c_struct(self) -> L.GmSystem:
        return L.GmSystem(self.n_structures, self.n_atoms, _ptr(self.atom_ptr), _ptr(self.pos), _ptr(self.species),
                          _ptr(self.cell), _ptr(self.pbc))


class NeighborList:
    """Device CSR neighbour list (the gm_nlist of the C ABI)."""

    def __init__(self, n_atoms, capacity, device="cuda"):
        dev = torch.device(device)
        self.capacity = int(capacity)
        self.row_ptr = torch.zeros(n_atoms + 1, dtype=torch.int32, device=dev)
        self.col = torch.zeros(max(self.capacity, 1), dtype=torch.int32, device=dev)
        self.shift = torch.zeros(max(self.capacity, 1), 4, dtype=torch.int8, device=dev)
        self.n_pairs = torch.zeros(1, dtype=torch.int64, device=dev)

    def c_struct(self) -> L.GmNlist:
        return L.GmNlist(self.capacity, _ptr(self.row_ptr), _ptr(self.col), _ptr(self.shift), _ptr(self.n_pairs))

    def triples(self):
        """Host copy as an int64 [P, 5] array (i, j, n0, n1, n2), sorted lexicographically."""
        rp = self.row_ptr.cpu().numpy().astype(np.int64)
        P = int(rp[-1])
        i = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
        t = np.column_stack([i, self.col[:P].cpu().numpy().astype(np.int64),
                             self.shift[:P, :3].cpu().numpy().astype(np.int64)])
        return t[np.lexsort(t.T[::-1])]


class MDParams:
    """Integration parameters (the gm_md_params of the C ABI).  Defaults: the paper's MD
    configuration (NVT, 0.5 fs, chain of 3 with 2 chain steps and 3 Suzuki-Yoshida steps,
    tau = 100 time steps, skin 0.5 A) at 600 K."""

    def __init__(self, dt=0.5, skin=0.5, temperature=600.0, tau=None, ensemble="nvt", chain_length=3,
                 chain_steps=2, sy_steps=3):
        self.dt, self.skin, self.temperature = float(dt), float(skin), float(temperature)
        self.tau = float(tau) if tau is not None else 100.0 * float(dt)
        self.ensemble, self.chain_length, self.chain_steps, self.sy_steps = ensemble, chain_length, chain_steps, sy_steps

    def c_struct(self) -> L.GmMdParams:
        return L.GmMdParams(self.dt, self.skin, self.temperature, self.tau,
                            L.GM_MD_NVT if self.ensemble == "nvt" else L.GM_MD_NVE, self.chain_length,
                            self.chain_steps, self.sy_steps)


class MDState:
    """Device buffers of an MD run (the gm_md_state of the C ABI).  The positions are the
    system's own (sysd.pos), integrated in place."""

    def __init__(self, sysd, masses_by_species, vel):
        dev = sysd.pos.device
        N, B = sysd.n_atoms, sysd.n_structures
        self.pos = sysd.pos
        self.vel = torch.as_tensor(np.asarray(vel, np.float64), device=dev).contiguous()
        self.mass = torch.as_tensor(np.asarray(masses_by_species, np.float64), device=dev).contiguous()
        self.forces = torch.zeros(N, 3, dtype=torch.float32, device=dev)
        self.energy = torch.zeros(B, dtype=torch.float64, device=dev)
        self.kinetic = torch.zeros(B, dtype=torch.float64, device=dev)
        self.pos_ref = torch.zeros_like(sysd.pos)
        self.chain = torch.zeros(B, 2, L.GM_MD_MAX_CHAIN, dtype=torch.float64, device=dev)
        self.n_builds = torch.zeros(1, dtype=torch.int64, device=dev)

    def c_struct(self) -> L.GmMdState:
        return L.GmMdState(_ptr(self.pos), _ptr(self.vel), _ptr(self.mass), _ptr(self.forces), _ptr(self.energy),
                           _ptr(self.kinetic), _ptr(self.pos_ref), _ptr(self.chain), _ptr(self.n_builds))


class GMNN:
    """A GMNN model on the GPU (handle to libgm's gm_model)."""

    def __init__(self, desc: dict, params=None, precision="fp32", device="cuda"):
        self.device = torch.device(device)
        self.desc = dict(desc)
        self.precision = precision
        self.n_ensemble = max(1, int(desc.get("n_ensemble", 1)))
        self.cdesc = L.GmModelDesc(int(desc["n_species"]), int(desc.get("n_basis", 7)), int(desc.get("n_radial", 5)),
                                   int(desc["n_hidden"]), ACT[desc.get("activation", "silu")], PREC[precision],
                                   float(desc.get("r_min", 0.5)), float(desc["r_cut"]),
                                   BASIS[desc.get("basis", "gaussian")], self.n_ensemble)
        self.n_param = L.gm_param_count(self.cdesc)
        with torch.cuda.device(self.device):
            self.handle = L.gm_model_create(self.cdesc)
        self.status = torch.zeros(1, dtype=torch.int32, device=self.device)
        self._ws = {}
        self.tuning = {}
        self.theta = None
        if params is not None:
            self.set_params(pack_theta(params))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                L.gm_model_destroy(h)
            except Exception:  # pragma: no cover
                pass
            self.handle = None

    # -------------------------------------------------------------- parameters
    def set_params(self, theta):
        th = torch.as_tensor(theta, dtype=torch.float32, device=self.device).contiguous()
        if th.numel() != self.n_param:
            raise ValueError(f"theta has {th.numel()} entries, expected {self.n_param}")
        self.theta = th
        L.gm_model_set_params(self.handle, _ptr(th), _stream())

    TUNING_KEYS = {"pair_tpa": L.GM_TUNE_PAIR_TPA, "split_mask": L.GM_TUNE_SPLIT_MASK, "gemm_bn": L.GM_TUNE_GEMM_BN,
                   "nl_mode": L.GM_TUNE_NL_MODE, "nl_split": L.GM_TUNE_NL_SPLIT, "nl_blocks": L.GM_TUNE_NL_BLOCKS,
                   "nl_two_pass": L.GM_TUNE_NL_TWO_PASS, "nl_items": L.GM_TUNE_NL_ITEMS,
                   "gemm_cps": L.GM_TUNE_GEMM_CPS, "pg_split_mask": L.GM_TUNE_PG_SPLIT_MASK,
                   "debug_stall": L.GM_TUNE_DEBUG_STALL, "f16_backward": L.GM_TUNE_F16_BACKWARD,
                   "fused_mlp": L.GM_TUNE_FUSED_MLP, "forces_tpa": L.GM_TUNE_FORCES_TPA,
                   "mlp_cluster": L.GM_TUNE_MLP_CLUSTER, "mlp_ctas": L.GM_TUNE_MLP_CTAS}

    def set_tuning(self, **knobs):
        """Speed knobs of the library (gm_model_set_tuning), by the names of TUNING_KEYS (the
        GM_TUNE_* keys of include/gm.h in lower case).  None leaves a knob unchanged."""
        for name, val in knobs.items():
            if name not in self.TUNING_KEYS:
                raise ValueError(f"unknown tuning knob {name!r}")
            if val is not None:
                L.gm_model_set_tuning(self.handle, self.TUNING_KEYS[name], int(val))
                self.tuning[name] = int(val)

    # -------------------------------------------------------------- buffers
    def workspace(self, op, sysd: DeviceSystem, capacity=0):
        need = L.gm_workspace_size(self.handle, sysd.n_structures, sysd.n_atoms, capacity, op)
        buf = self._ws.get(op)
        if buf is None or buf.numel() < need:
            buf = torch.empty(need, dtype=torch.uint8, device=self.device)
            self._ws[op] = buf
        return _ptr(buf), int(buf.numel())

    def estimate_capacity(self, sysd: DeviceSystem, margin=1.3, r_list=None):
        rc = float(self.desc["r_cut"]) if r_list is None else float(r_list)
        vols = np.abs(np.linalg.det(sysd.host_cells))
        n = sysd.host_counts.astype(np.float64)
        est = np.sum(n * n / vols * 4.0 / 3.0 * math.pi * rc ** 3)
        return int(est * margin) + 64 * sysd.n_structures + 1024

    def clear_status(self):
        L.gm_status_clear(_ptr(self.status), _stream())

    def read_status(self) -> int:
        torch.cuda.current_stream().synchronize()
        return int(self.status.item())

    def check_status(self, where="device"):
        code = self.read_status()
        if code != L.GM_OK:
            raise L.GmError(code, where)

    # -------------------------------------------------------------- operations
    def build_neighbors(self, sysd: DeviceSystem, nl: NeighborList | None = None, check=True) -> NeighborList:
        """Cell-list neighbour search.  With check=True, reads the status and grows the
        capacity (and retries) on overflow."""
        if nl is None:
            nl = NeighborList(sysd.n_atoms, self.estimate_capacity(sysd), self.device)
        for _ in range(3):
            ws, wsb = self.workspace(L.GM_OP_NEIGHBORS, sysd, nl.capacity)
            self.clear_status()
            L.gm_build_neighbors(self.handle, sysd.c_struct(), nl.c_struct(), ws, wsb, _ptr(self.status), _stream())
            if not check:
                return nl
            code = self.read_status()
            if code == L.GM_OK:
                return nl
            if code != L.GM_ERR_CAPACITY:
                raise L.GmError(code, "gm_build_neighbors (device)")
            need = int(nl.n_pairs.item())
            nl = NeighborList(sysd.n_atoms, int(need * 1.2) + 1024, self.device)
        raise RuntimeError("neighbour list capacity retries exhausted")

    def energy_forces(self, sysd: DeviceSystem, nl: NeighborList, virial=False, out=None, clear=True):
        """(E [B] float64, F [N,3] float32, W [B,3,3] float64 or None) on the device."""
        if out is None:
            E = torch.empty(sysd.n_structures, dtype=torch.float64, device=self.device)
            F = torch.empty(sysd.n_atoms, 3, dtype=torch.float32, device=self.device)
            W = torch.empty(sysd.n_structures, 3, 3, dtype=torch.float64, device=self.device) if virial else None
        else:
            E, F, W = out
        ws, wsb = self.workspace(L.GM_OP_ENERGY_FORCES, sysd, nl.capacity)
        if clear:
            self.clear_status()
        L.gm_energy_forces(self.handle, sysd.c_struct(), nl.c_struct(), _ptr(E), _ptr(F), _ptr(W), ws, wsb,
                           _ptr(self.status), _stream())
        return E, F, W

    def energy_forces_ensemble(self, sysd: DeviceSystem, nl: NeighborList, mode="mean", virial=False):
        """Shallow ensemble (n_ensemble > 1): a dict with the mean energy "E" [B] and forces
        "F" [N,3] (gradient of the mean energy), "E_heads" [B,E], "E_std" [B] and, in the
        Jacobian mode, "F_heads" [E,N,3] and "F_std" [N]; "W" [B,3,3] with virial=True."""
        E_ = self.n_ensemble
        dev = self.device
        B, N = sysd.n_structures, sysd.n_atoms
        out = {"E": torch.empty(B, dtype=torch.float64, device=dev), "F": torch.empty(N, 3, dtype=torch.float32, device=dev),
               "E_heads": torch.empty(B, E_, dtype=torch.float64, device=dev),
               "E_std": torch.empty(B, dtype=torch.float64, device=dev),
               "W": torch.empty(B, 3, 3, dtype=torch.float64, device=dev) if virial else None}
        jac = mode == "jacobian"
        if jac:
            out["F_heads"] = torch.empty(E_, N, 3, dtype=torch.float32, device=dev)
            out["F_std"] = torch.empty(N, dtype=torch.float32, device=dev)
        ws, wsb = self.workspace(L.GM_OP_ENERGY_FORCES, sysd, nl.capacity)
        self.clear_status()
        L.gm_energy_forces_ensemble(self.handle, sysd.c_struct(), nl.c_struct(), _ptr(out["E"]), _ptr(out["F"]),
                                    _ptr(out["W"]), _ptr(out["E_heads"]), _ptr(out["E_std"]),
                                    L.GM_ENS_JACOBIAN if jac else L.GM_ENS_MEAN_GRADIENT,
                                    _ptr(out.get("F_heads")), _ptr(out.get("F_std")), ws, wsb, _ptr(self.status),
                                    _stream())
        return out

    # -------------------------------------------------------------- molecular dynamics
    def md_neighbor_list(self, sysd: DeviceSystem, params: MDParams, margin=1.5):
        """An empty neighbour list with room for the skin list (pairs within r_cut + skin)."""
        cap = self.estimate_capacity(sysd, margin, float(self.desc["r_cut"]) + params.skin)
        return NeighborList(sysd.n_atoms, cap, self.device)

    def md_init(self, sysd: DeviceSystem, nl: NeighborList, params: MDParams, state: MDState, clear=True):
        ws, wsb = self.workspace(L.GM_OP_MD, sysd, nl.capacity)
        if clear:
            self.clear_status()
        L.gm_md_init(self.handle, sysd.c_struct(), nl.c_struct(), params.c_struct(), state.c_struct(), ws, wsb,
                     _ptr(self.status), _stream())

    def md_run(self, sysd: DeviceSystem, nl: NeighborList, params: MDParams, state: MDState, n_steps: int):
        """n_steps MD steps on the current stream (no host synchronisation)."""
        ws, wsb = self.workspace(L.GM_OP_MD, sysd, nl.capacity)
        L.gm_md_run(self.handle, sysd.c_struct(), nl.c_struct(), params.c_struct(), state.c_struct(), int(n_steps),
                    ws, wsb, _ptr(self.status), _stream())

    def capture_md(self, sysd: DeviceSystem, nl: NeighborList, params: MDParams, state: MDState, n_steps: int):
        """CUDA graph of md_run(n_steps) on fixed buffers (the paper's compiled inner steps)."""
        self.workspace(L.GM_OP_MD, sysd, nl.capacity)
        torch.cuda.current_stream().synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self.md_run(sysd, nl, params, state, n_steps)
        return graph

    def step(self, sysd: DeviceSystem, nl: NeighborList, out):
        """One MD-style step on the current stream: clear the status word, rebuild the
        neighbour list into nl (fixed capacity) and evaluate energies and forces into out."""
        self.clear_status()
        self.build_neighbors(sysd, nl, check=False)
        return self.energy_forces(sysd, nl, out=out, clear=False)

    def capture_step(self, sysd: DeviceSystem, nl: NeighborList, out):
        """CUDA graph of step() for fixed buffers (sysd.pos, nl, out, the workspaces).
        Replay it after writing new positions into sysd.pos.  With library stage timing on
        while capturing, the stage events become record nodes of the graph: read them with
        gm_profile_collect after each replay."""
        side = torch.cuda.Stream(device=self.device)
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.step(sysd, nl, out)       # warm: workspaces, kernel attributes, tensor maps
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.current_stream().synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self.step(sysd, nl, out)
        return graph

    def descriptors(self, sysd: DeviceSystem, nl: NeighborList, features=True):
        psi = torch.empty(sysd.n_atoms, 5, 20, dtype=torch.float32, device=self.device)
        G = torch.empty(sysd.n_atoms, 360, dtype=torch.float32, device=self.device) if features else None
        ws, wsb = self.workspace(L.GM_OP_ENERGY_FORCES, sysd, nl.capacity)
        self.clear_status()
        L.gm_descriptors(self.handle, sysd.c_struct(), nl.c_struct(), _ptr(psi), _ptr(G), ws, wsb, _ptr(self.status),
                         _stream())
        return psi, G

    def param_grad(self, sysd: DeviceSystem, nl: NeighborList, dL_dE, dL_dF, clear=True):
        g = torch.empty(self.n_param, dtype=torch.float32, device=self.device)
        ws, wsb = self.workspace(L.GM_OP_PARAM_GRAD, sysd, nl.capacity)
        if clear:
            self.clear_status()
        L.gm_param_grad(self.handle, sysd.c_struct(), nl.c_struct(), _ptr(dL_dE.contiguous()),
                        _ptr(dL_dF.contiguous()), _ptr(g), ws, wsb, _ptr(self.status), _stream())
        return g

    def force_matching_loss(self, sysd: DeviceSystem, E, E_ref, F, F_ref, w_energy=1.0, w_forces=1.0):
        loss = torch.empty(1, dtype=torch.float64, device=self.device)
        gE = torch.empty(sysd.n_structures, dtype=torch.float64, device=self.device)
        gF = torch.empty(sysd.n_atoms, 3, dtype=torch.float32, device=self.device)
        L.gm_force_matching_loss(sysd.c_struct(), _ptr(E), _ptr(E_ref), _ptr(F), _ptr(F_ref), float(w_energy),
                                 float(w_forces), _ptr(loss), _ptr(gE), _ptr(gF), _ptr(self.status), _stream())
        return loss, gE, gF


class GMNNFunction(torch.autograd.Function):
    """(E, F) = GMNNFunction.apply(theta, model, sysd, nl).

    Backward returns d/dtheta of sum_b gE_b E_b + sum_i gF_i . F_i through
    gm_param_grad (hand-written force double-backward kernels); positions get no
    gradient."""

    @staticmethod
    def forward(ctx, theta, model: GMNN, sysd: DeviceSystem, nl: NeighborList):
        # repack on every call: an optimiser updates theta in place (same storage, new
        # values), so the storage address says nothing about whether the weights changed
        model.set_params(theta.detach())
        E, F, _ = model.energy_forces(sysd, nl)
        ctx.model, ctx.sysd, ctx.nl = model, sysd, nl
        return E, F

    @staticmethod
    def backward(ctx, gE, gF):
        if gE is None:
            gE = torch.zeros(ctx.sysd.n_structures, dtype=torch.float64, device=ctx.model.device)
        if gF is None:
            gF = torch.zeros(ctx.sysd.n_atoms, 3, dtype=torch.float32, device=ctx.model.device)
        g = ctx.model.param_grad(ctx.sysd, ctx.nl, gE.to(torch.float64), gF.to(torch.float32))
        return g, None, None, None
