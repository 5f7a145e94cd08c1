"""ctypes declarations of libgm (include/gm.h), with the same function names.

Argument marshalling only: every entry point takes plain integers (device pointers, sizes,
the CUDA stream handle) and ctypes structs; no computation happens here.  A missing or
unloadable libgm.so raises immediately -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

LIB_PATH = Path(__file__).resolve().parent / "libgm.so"

GM_OK, GM_ERR_ARG, GM_ERR_CAPACITY, GM_ERR_UNSUPPORTED, GM_ERR_CUDA, GM_ERR_TIMEOUT, GM_ERR_SPECIES, \
    GM_ERR_WORKSPACE = range(8)
GM_ACT_TANH, GM_ACT_SILU = 0, 1
GM_PREC_FP32, GM_PREC_MIXED = 0, 1
GM_BASIS_GAUSSIAN, GM_BASIS_BESSEL = 0, 1
GM_ENS_MEAN_GRADIENT, GM_ENS_JACOBIAN = 0, 1
GM_MD_NVE, GM_MD_NVT = 0, 1
GM_MD_MAX_CHAIN = 8
GM_MAX_ENSEMBLE = 32
GM_OP_NEIGHBORS, GM_OP_ENERGY_FORCES, GM_OP_PARAM_GRAD, GM_OP_MD = 0, 1, 2, 3
GM_MAX_ATOMS = 4_000_000
MIXED_AVAILABLE = True   # GM_PREC_MIXED: BF16 network GEMMs on tcgen05

STATUS_NAMES = {0: "GM_OK", 1: "GM_ERR_ARG", 2: "GM_ERR_CAPACITY", 3: "GM_ERR_UNSUPPORTED", 4: "GM_ERR_CUDA",
                5: "GM_ERR_TIMEOUT", 6: "GM_ERR_SPECIES", 7: "GM_ERR_WORKSPACE"}

# every exported symbol of include/gm.h
EXPORTS = ("gm_param_count", "gm_model_create", "gm_model_set_params", "gm_model_destroy", "gm_workspace_size",
           "gm_build_neighbors", "gm_energy_forces", "gm_param_grad", "gm_force_matching_loss", "gm_descriptors",
           "gm_status_clear", "gm_status_string", "gm_last_error", "gm_profile_enable", "gm_profile_reset",
           "gm_profile_n_stages", "gm_profile_stage_name", "gm_profile_collect", "gm_build_neighbors_noalloc", "gm_model_set_tuning",
           "gm_profile_forget_graphs", "gm_model_pair_lanes", "gm_model_device_bytes", "gm_probe_alu",
           "gm_energy_forces_ensemble", "gm_md_init", "gm_md_run", "gm_model_force_lanes")


class GmModelDesc(ctypes.Structure):
    _fields_ = [("n_species", ctypes.c_int32), ("n_basis", ctypes.c_int32), ("n_radial", ctypes.c_int32),
                ("n_hidden", ctypes.c_int32), ("activation", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("r_min", ctypes.c_double), ("r_cut", ctypes.c_double), ("basis", ctypes.c_int32),
                ("n_ensemble", ctypes.c_int32)]


class GmSystem(ctypes.Structure):
    _fields_ = [("n_structures", ctypes.c_int32), ("n_atoms", ctypes.c_int32), ("atom_ptr", ctypes.c_void_p),
                ("pos", ctypes.c_void_p), ("species", ctypes.c_void_p), ("cell", ctypes.c_void_p),
                ("pbc", ctypes.c_void_p)]


class GmNlist(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int64), ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("shift", ctypes.c_void_p), ("n_pairs", ctypes.c_void_p)]


class GmMdParams(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("skin", ctypes.c_double), ("temperature", ctypes.c_double),
                ("tau", ctypes.c_double), ("ensemble", ctypes.c_int32), ("chain_length", ctypes.c_int32),
                ("chain_steps", ctypes.c_int32), ("sy_steps", ctypes.c_int32)]


class GmMdState(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_void_p), ("vel", ctypes.c_void_p), ("mass", ctypes.c_void_p),
                ("forces", ctypes.c_void_p), ("energy", ctypes.c_void_p), ("kinetic", ctypes.c_void_p),
                ("pos_ref", ctypes.c_void_p), ("chain", ctypes.c_void_p), ("n_builds", ctypes.c_void_p)]


class GmError(RuntimeError):
    def __init__(self, code, where, detail=""):
        self.code = code
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)} {detail}".strip())


_lib = None
_P = ctypes.c_void_p


def load():
    """Load libgm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2505_22168_b300.build`")
    lib = ctypes.CDLL(str(LIB_PATH))
    st = ctypes.c_int
    sig = {
        "gm_param_count": (ctypes.c_int64, [ctypes.POINTER(GmModelDesc)]),
        "gm_model_create": (st, [ctypes.POINTER(GmModelDesc), ctypes.POINTER(_P)]),
        "gm_model_set_params": (st, [_P, _P, _P]),
        "gm_model_destroy": (None, [_P]),
        "gm_workspace_size": (st, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                   ctypes.POINTER(ctypes.c_size_t)]),
        "gm_build_neighbors": (st, [_P, ctypes.POINTER(GmSystem), ctypes.POINTER(GmNlist), _P, ctypes.c_size_t, _P, _P]),
        "gm_energy_forces": (st, [_P, ctypes.POINTER(GmSystem), ctypes.POINTER(GmNlist), _P, _P, _P, _P,
                                  ctypes.c_size_t, _P, _P]),
        "gm_param_grad": (st, [_P, ctypes.POINTER(GmSystem), ctypes.POINTER(GmNlist), _P, _P, _P, _P,
                               ctypes.c_size_t, _P, _P]),
        "gm_force_matching_loss": (st, [ctypes.POINTER(GmSystem), _P, _P, _P, _P, ctypes.c_double, ctypes.c_double,
                                        _P, _P, _P, _P, _P]),
        "gm_descriptors": (st, [_P, ctypes.POINTER(GmSystem), ctypes.POINTER(GmNlist), _P, _P, _P, ctypes.c_size_t,
                                _P, _P]),
        "gm_status_clear": (st, [_P, _P]),
        "gm_status_string": (ctypes.c_char_p, [st]),
        "gm_last_error": (ctypes.c_char_p, []),
        "gm_profile_enable": (None, [ctypes.c_int]),
        "gm_profile_reset": (None, []),
        "gm_profile_n_stages": (ctypes.c_int, []),
        "gm_profile_stage_name": (ctypes.c_char_p, [ctypes.c_int]),
        "gm_profile_collect": (st, [_P, _P, ctypes.c_int, _P]),
        "gm_build_neighbors_noalloc": (st, [_P, ctypes.POINTER(GmSystem), ctypes.POINTER(GmNlist), _P, _P]),
        "gm_model_set_tuning": (st, [_P, ctypes.c_int32, ctypes.c_int32]),
        "gm_profile_forget_graphs": (None, []),
        "gm_model_pair_lanes": (ctypes.c_int32, [_P, ctypes.c_int32]),
        "gm_model_force_lanes": (ctypes.c_int32, [_P, ctypes.c_int32]),
        "gm_model_device_bytes": (ctypes.c_size_t, [_P]),
        "gm_probe_alu": (st, [ctypes.c_int32, ctypes.c_int64, _P, ctypes.POINTER(ctypes.c_double), _P]),
        "gm_md_init": (st, [_P, ctypes.POINTER(GmSystem), ctypes.POINTER(GmNlist), ctypes.POINTER(GmMdParams),
                            ctypes.POINTER(GmMdState), _P, ctypes.c_size_t, _P, _P]),
        "gm_md_run": (st, [_P, ctypes.POINTER(GmSystem), ctypes.POINTER(GmNlist), ctypes.POINTER(GmMdParams),
                           ctypes.POINTER(GmMdState), ctypes.c_int32, _P, ctypes.c_size_t, _P, _P]),
        "gm_energy_forces_ensemble": (st, [_P, ctypes.POINTER(GmSystem), ctypes.POINTER(GmNlist), _P, _P, _P, _P, _P,
                                           ctypes.c_int32, _P, _P, _P, ctypes.c_size_t, _P, _P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def check(code, where):
    """Raise GmError for a non-zero synchronous status."""
    if code != GM_OK:
        detail = load().gm_last_error().decode()
        raise GmError(code, where, detail)


# thin wrappers with the C names ------------------------------------------------------

def gm_param_count(desc: GmModelDesc) -> int:
    return int(load().gm_param_count(ctypes.byref(desc)))


def gm_model_create(desc: GmModelDesc) -> int:
    h = _P()
    check(load().gm_model_create(ctypes.byref(desc), ctypes.byref(h)), "gm_model_create")
    return h.value


def gm_model_set_params(model: int, theta_ptr: int, stream: int):
    check(load().gm_model_set_params(model, theta_ptr, stream), "gm_model_set_params")


GM_TUNE_PAIR_TPA, GM_TUNE_SPLIT_MASK, GM_TUNE_GEMM_BN = 0, 1, 2
GM_TUNE_NL_MODE, GM_TUNE_NL_SPLIT, GM_TUNE_NL_BLOCKS, GM_TUNE_NL_TWO_PASS, GM_TUNE_NL_ITEMS = 3, 4, 5, 6, 7
GM_TUNE_GEMM_CPS = 8
GM_TUNE_PG_SPLIT_MASK = 9
GM_TUNE_DEBUG_STALL = 10
GM_TUNE_F16_BACKWARD = 11
GM_TUNE_FUSED_MLP = 12
GM_TUNE_FORCES_TPA = 13
GM_TUNE_MLP_CLUSTER = 14
GM_TUNE_MLP_CTAS = 15
GM_NL_MODE_AUTO, GM_NL_MODE_PHASES = 0, 1


def gm_model_set_tuning(model: int, key: int, value: int):
    check(load().gm_model_set_tuning(model, key, value), "gm_model_set_tuning")


def gm_model_pair_lanes(model: int, n_atoms: int) -> int:
    return int(load().gm_model_pair_lanes(model, n_atoms))


def gm_model_force_lanes(model: int, n_atoms: int) -> int:
    return int(load().gm_model_force_lanes(model, n_atoms))


def gm_model_device_bytes(model: int) -> int:
    return int(load().gm_model_device_bytes(model))


def gm_probe_alu(kind: int, iters: int, sink: int, stream: int) -> float:
    """Launch the throughput probe; returns the operations launched (see gm.h)."""
    ops = ctypes.c_double(0.0)
    check(load().gm_probe_alu(kind, iters, sink, ctypes.byref(ops), stream), "gm_probe_alu")
    return float(ops.value)


def gm_model_destroy(model: int):
    load().gm_model_destroy(model)


def gm_workspace_size(model: int, n_structures: int, n_atoms: int, capacity: int, op: int) -> int:
    out = ctypes.c_size_t(0)
    check(load().gm_workspace_size(model, n_structures, n_atoms, capacity, op, ctypes.byref(out)),
          "gm_workspace_size")
    return int(out.value)


def gm_build_neighbors(model, sys: GmSystem, nl: GmNlist, ws, ws_bytes, status, stream):
    check(load().gm_build_neighbors(model, ctypes.byref(sys), ctypes.byref(nl), ws, ws_bytes, status, stream),
          "gm_build_neighbors")


def gm_build_neighbors_noalloc(model, sys: GmSystem, nl: GmNlist, status, stream):
    """Neighbour build without a workspace (fixed scratch inside the library; see gm.h)."""
    check(load().gm_build_neighbors_noalloc(model, ctypes.byref(sys), ctypes.byref(nl), status, stream),
          "gm_build_neighbors_noalloc")


def gm_energy_forces(model, sys: GmSystem, nl: GmNlist, energy, forces, virial, ws, ws_bytes, status, stream):
    check(load().gm_energy_forces(model, ctypes.byref(sys), ctypes.byref(nl), energy, forces, virial, ws, ws_bytes,
                                  status, stream), "gm_energy_forces")


def gm_energy_forces_ensemble(model, sys: GmSystem, nl: GmNlist, energy, forces, virial, energy_heads, energy_std,
                              mode, forces_heads, force_std, ws, ws_bytes, status, stream):
    check(load().gm_energy_forces_ensemble(model, ctypes.byref(sys), ctypes.byref(nl), energy, forces, virial,
                                           energy_heads, energy_std, mode, forces_heads, force_std, ws, ws_bytes,
                                           status, stream), "gm_energy_forces_ensemble")


def gm_md_init(model, sys: GmSystem, nl: GmNlist, params: GmMdParams, state: GmMdState, ws, ws_bytes, status,
               stream):
    check(load().gm_md_init(model, ctypes.byref(sys), ctypes.byref(nl), ctypes.byref(params), ctypes.byref(state),
                            ws, ws_bytes, status, stream), "gm_md_init")


def gm_md_run(model, sys: GmSystem, nl: GmNlist, params: GmMdParams, state: GmMdState, n_steps, ws, ws_bytes,
              status, stream):
    check(load().gm_md_run(model, ctypes.byref(sys), ctypes.byref(nl), ctypes.byref(params), ctypes.byref(state),
                           n_steps, ws, ws_bytes, status, stream), "gm_md_run")


def gm_param_grad(model, sys: GmSystem, nl: GmNlist, dL_dE, dL_dF, grad_theta, ws, ws_bytes, status, stream):
    check(load().gm_param_grad(model, ctypes.byref(sys), ctypes.byref(nl), dL_dE, dL_dF, grad_theta, ws, ws_bytes,
                               status, stream), "gm_param_grad")


def gm_force_matching_loss(sys: GmSystem, energy, energy_ref, forces, forces_ref, w_energy, w_forces, loss, dL_dE,
                           dL_dF, status, stream):
    check(load().gm_force_matching_loss(ctypes.byref(sys), energy, energy_ref, forces, forces_ref, w_energy, w_forces,
                                        loss, dL_dE, dL_dF, status, stream), "gm_force_matching_loss")


def gm_descriptors(model, sys: GmSystem, nl: GmNlist, psi, features, ws, ws_bytes, status, stream):
    check(load().gm_descriptors(model, ctypes.byref(sys), ctypes.byref(nl), psi, features, ws, ws_bytes, status,
                                stream), "gm_descriptors")


def gm_status_clear(status, stream):
    check(load().gm_status_clear(status, stream), "gm_status_clear")


def gm_status_string(code: int) -> str:
    return load().gm_status_string(code).decode()


def gm_profile_enable(on: bool):
    load().gm_profile_enable(1 if on else 0)


def gm_profile_reset():
    load().gm_profile_reset()


def gm_profile_forget_graphs():
    load().gm_profile_forget_graphs()


def gm_profile_collect():
    """({stage name: (total ms, count)}, kernel launches since the last reset)."""
    lib = load()
    n = lib.gm_profile_n_stages()
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int64 * n)()
    launches = ctypes.c_int64(0)
    check(lib.gm_profile_collect(ctypes.addressof(ms), ctypes.addressof(cnt), n, ctypes.addressof(launches)),
          "gm_profile_collect")
    stages = {lib.gm_profile_stage_name(q).decode(): (ms[q], cnt[q]) for q in range(n)}
    return stages, int(launches.value)
