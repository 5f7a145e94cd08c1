"""Launch-shape autotuner for one energy-and-forces step.

The library's tuning knobs (gm_model_set_tuning) change how the kernels are launched, not
what they compute: the neighbour search's work items and parts per cell (the list is the same
bit for bit), the lanes per atom of the pair kernels and the tensor-core tile width (energies
and forces change only by the order of FP32 summation).  The tuner captures the step as a CUDA graph for
each candidate setting, times replays with CUDA events, and keeps the fastest setting by
coordinate descent over the knobs (one knob at a time, the others at their best so far).
Results can be cached in a JSON file keyed by device, system shape and model.
"""
from __future__ import annotations

import json
import os
from pathlib import Path

import torch

# candidate values per knob, tried in this order (0 = the library's own choice)
SPACE = {
    "nl_items": (0, 1, 2),
    "nl_split": (0, 1, 2, 4, 8, 16),
    "pair_tpa": (0, 1, 4, 8, 32),
    "forces_tpa": (0, 8, 16, 32),
    "gemm_bn": (0, 64, 128, 256),
    "gemm_cps": (0, 1, 2),
    "mlp_cluster": (0, 1, 2, 4, 8),
}


def _key(model, sysd, nl) -> str:
    dev = torch.cuda.get_device_name(model.device)
    d = model.desc
    return (f"{dev}|N={sysd.n_atoms}|B={sysd.n_structures}|cap={nl.capacity}|H={d['n_hidden']}|S={d['n_species']}"
            f"|rc={d['r_cut']}|{model.precision}")


def time_step(model, sysd, nl, out, reps=20, warmup=3) -> float:
    """Milliseconds per replay of the captured step (neighbour build + energies and forces)."""
    graph = model.capture_step(sysd, nl, out)
    for _ in range(warmup):
        graph.replay()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stream.synchronize()
    e0.record(stream)
    for _ in range(reps):
        graph.replay()
    e1.record(stream)
    e1.synchronize()
    if model.read_status() != 0:
        raise RuntimeError(f"device status {model.read_status()} while tuning")
    del graph
    return e0.elapsed_time(e1) / reps


def tune(model, sysd, nl, out, reps=20, cache: str | os.PathLike | None = None, space=None, log=None,
         timer=None, key=None) -> dict:
    """Pick the fastest knob settings for this model and system; returns
    {"settings": {...}, "ms": best, "default_ms": ms with all knobs 0, "trials": [...]}.
    The model keeps the chosen settings.  `timer(model)` replaces the graph timing (tests)."""
    space = dict(SPACE if space is None else space)
    if model.precision != "mixed":
        space.pop("gemm_bn", None)            # the FP32 path has no tensor-core tiles
        space.pop("gemm_cps", None)
        space.pop("mlp_cluster", None)
    if timer is None:
        def timer(m):
            return time_step(m, sysd, nl, out, reps)
    if key is None:
        key = _key(model, sysd, nl)
    if cache is not None and Path(cache).exists():
        table = json.loads(Path(cache).read_text())
        if key in table:
            hit = table[key]
            model.set_tuning(**hit["settings"])
            return dict(hit, cached=True)
    best = {k: 0 for k in space}
    model.set_tuning(**best)
    best_ms = timer(model)
    default_ms = best_ms
    trials = [(dict(best), best_ms)]
    for knob, values in space.items():
        for v in values:
            if v == best[knob]:
                continue
            trial = dict(best, **{knob: v})
            model.set_tuning(**trial)
            ms = timer(model)
            trials.append((trial, ms))
            if log:
                log(f"tune {trial} {ms:.4f} ms")
            if ms < best_ms:
                best, best_ms = trial, ms
        model.set_tuning(**best)
    result = {"settings": best, "ms": best_ms, "default_ms": default_ms, "trials": trials}
    if cache is not None:
        path = Path(cache)
        table = json.loads(path.read_text()) if path.exists() else {}
        table[key] = {"settings": best, "ms": best_ms, "default_ms": default_ms}
        path.write_text(json.dumps(table, indent=1, sort_keys=True))
    return dict(result, cached=False)
