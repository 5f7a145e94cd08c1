#!/usr/bin/env python
"""Energy+force throughput of the B300 GMNN path (atom-steps/s).

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

One step = the whole hot path on one batch: cell-list neighbour rebuild, moments,
contractions, network forward and backward, forces, FP64 energy/virial reductions.
Headline workload: the 1536-atom EMIM+BF4- box (64 ion pairs, r_cut 6 A, MLP 2x512)
with a seeded 0.01 A random walk of the positions every step; the 131,072-atom Li3PO4
box is reported under "variants".  Each timed step is bracketed by CUDA events on the
library's stream; a 256 MiB buffer is written between timed steps (outside the events)
to flush L2.  Under torchrun every rank runs its own replica (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "energy+force atom-steps/s at 1.5k & 131k atoms; mixed vs plain FP32 path"
UNIT = "atom-steps/s"
FP32_ALU_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12   # 148 SMs x 128 FP32 lanes x FMA x 2.032 GHz
FLUSH_BYTES = 256 << 20
# algorithmic work per unit (the measurement section of the scope table): the neighbour build
# moves 56 B per atom and 7 B per pair; the moments pass is ~160 FMA per pair, the force pass
# ~350 FMA per pair (2 flop each)
NL_BYTES_PER_ATOM, NL_BYTES_PER_PAIR = 56.0, 7.0
MOMENTS_FLOP_PER_PAIR, FORCES_FLOP_PER_PAIR = 320.0, 700.0


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ----------------------------------------------------------------------------- workloads

WORKLOADS = {
    2: "emim-64pairs-1536 (EMIM+BF4- box, 1536 atoms, L=25.43 A, r_cut 6 A, MLP 2x512, 0.01 A jitter/step)",
    3: "li3po4-batch-256 (256 Li3PO4-like boxes of 32-512 atoms, 67768 atoms, r_cut 5 A, MLP 2x256)",
    5: "li3po4-131072 (Li3PO4-like crystal, 131072 atoms, L=109.49 A, r_cut 6 A, MLP 2x512)",
}


def jitter_path(batch, seed, steps, sigma=0.01):
    """Positions for `steps` consecutive steps of a seeded random walk (host, FP64)."""
    rng = np.random.default_rng([seed, 51])
    pos = np.empty((steps,) + batch.pos.shape)
    cur = batch.pos.copy()
    for k in range(steps):
        cur = cur + rng.normal(0.0, sigma, cur.shape)
        pos[k] = cur
    return pos


# ----------------------------------------------------------------------------- clocks

class _Nvml:
    """Read-only NVML queries through ctypes (libnvidia-ml ships with the driver)."""

    CLOCK_SM = 1

    def __init__(self):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        rc = self.lib.nvmlInit_v2()
        if rc != 0:
            raise RuntimeError(f"nvmlInit_v2 returned {rc}")

    def handle(self, uuid, index):
        ct = self.ct
        h = ct.c_void_p()
        if uuid and self.lib.nvmlDeviceGetHandleByUUID(ct.c_char_p(uuid.encode()), ct.byref(h)) == 0:
            return h
        if self.lib.nvmlDeviceGetHandleByIndex_v2(ct.c_uint(index), ct.byref(h)) == 0:
            return h
        raise RuntimeError("no NVML handle")

    def clock(self, h):
        v = self.ct.c_uint()
        return v.value if self.lib.nvmlDeviceGetClockInfo(h, self.CLOCK_SM, self.ct.byref(v)) == 0 else None

    def max_clock(self, h):
        v = self.ct.c_uint()
        return v.value if self.lib.nvmlDeviceGetMaxClockInfo(h, self.CLOCK_SM, self.ct.byref(v)) == 0 else None

    def reasons(self, h):
        v = self.ct.c_ulonglong()
        for name in ("nvmlDeviceGetCurrentClocksEventReasons", "nvmlDeviceGetCurrentClocksThrottleReasons"):
            f = getattr(self.lib, name, None)
            if f is not None and f(h, self.ct.byref(v)) == 0:
                return v.value
        return 0

    def power_w(self, h):
        v = self.ct.c_uint()
        return v.value / 1000.0 if self.lib.nvmlDeviceGetPowerUsage(h, self.ct.byref(v)) == 0 else None


_SAMPLER_CHILD = r"""
import sys, time, select
sys.path.insert(0, sys.argv[3])
from bench import _Nvml
nv = _Nvml()
h = nv.handle(sys.argv[1], int(sys.argv[2]))
print("max", nv.max_clock(h), flush=True)
while True:
    print("s", time.monotonic(), nv.clock(h), nv.reasons(h), nv.power_w(h), flush=True)
    r, _, _ = select.select([sys.stdin], [], [], 0.001)
    if r:
        break
"""


# end-to-end steps (host copies and a synchronisation each): enough wall time (~30 ms) that
# host jitter averages out
E2E_STEPS = 200


class ClockSampler:
    """SM clock, power and clock-event reasons sampled about every 1 ms through NVML (read
    only) by a child process while the timed region runs (no contention with the launch
    loop).  The region starts once the child has taken its first sample; samples carry the
    child's monotonic time and the summary keeps those inside the region, plus the first one
    after it when the region is shorter than the sampling interval."""

    REASONS = {"hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40,
               "sw_power_cap": 0x4}

    def __init__(self, torch_device=0):
        self.proc = None
        self.lines = []
        self.error = None
        self.t0 = self.t1 = None
        self.uuid, self.index = "", torch_device
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(torch_device).uuid)
            self.uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        except Exception as exc:
            self.error = f"{type(exc).__name__}: {exc}"

    def __enter__(self):
        try:
            self.proc = subprocess.Popen([sys.executable, "-c", _SAMPLER_CHILD, self.uuid, str(self.index), str(ROOT)],
                                         stdin=subprocess.PIPE, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                         text=True)
            while True:                               # wait until sampling has started
                line = self.proc.stdout.readline()
                if not line:
                    break
                self.lines.append(line)
                if line.startswith("s "):
                    break
            self.t0 = time.monotonic()
        except Exception as exc:
            self.error = f"{type(exc).__name__}: {exc}"
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is None:
            return
        self.t1 = time.monotonic()
        time.sleep(0.03)                              # let a sample after the region land
        try:
            out, err = self.proc.communicate(input="stop\n", timeout=10)
            self.lines += out.splitlines()
            if err.strip():
                self.error = err.strip().splitlines()[-1]
        except Exception as exc:
            self.proc.kill()
            self.error = f"{type(exc).__name__}: {exc}"

    def summary(self):
        max_mhz, clks, reasons, powers = None, [], set(), []
        for line in self.lines:
            p = line.split()
            if not p:
                continue
            if p[0] == "max" and len(p) > 1 and p[1] != "None":
                max_mhz = int(p[1])
        samples = []
        for line in self.lines:
            p = line.split()
            if len(p) >= 5 and p[0] == "s" and p[2] != "None":
                samples.append((float(p[1]), int(p[2]), int(p[3]), None if p[4] == "None" else float(p[4])))
        if self.t0 is not None and self.t1 is not None:
            inside = [s for s in samples if self.t0 <= s[0] <= self.t1]
            after = [s for s in samples if s[0] > self.t1][:1]
            samples = inside if len(inside) >= 2 else inside + after
        for _, clk, r, pw in samples:
            clks.append(clk)
            reasons |= {name for name, bit in self.REASONS.items() if r & bit}
            if pw is not None:
                powers.append(pw)
        if not clks:
            return {"sm_mhz": None, "sm_max_mhz": max_mhz, "reasons": ["unavailable"], "samples": 0,
                    "error": self.error}
        return {"sm_mhz": statistics.median(clks), "sm_max_mhz": max_mhz, "reasons": sorted(reasons),
                "samples": len(clks), "power_w_max": max(powers) if powers else None, "source": "NVML"}


# ----------------------------------------------------------------------------- roofline

def algorithmic_work(stage, n_atoms, n_pairs, H):
    """(amount, unit) of algorithmic work of one launch of a stage."""
    F = 360
    if stage == "gemm_l1" or stage == "gemm_b0":
        return 2.0 * n_atoms * F * H, "flop"
    if stage == "gemm_l2" or stage == "gemm_b1":
        return 2.0 * n_atoms * H * H, "flop"
    if stage == "mlp_fused":
        # the four layers in one kernel: L1 and B0 (360 x H each), L2 and B1 (H x H each)
        return 2.0 * n_atoms * (2 * F * H + 2 * H * H), "flop"
    if stage == "moments":
        return MOMENTS_FLOP_PER_PAIR * n_pairs, "flop"
    if stage == "forces":
        return FORCES_FLOP_PER_PAIR * n_pairs, "flop"
    if stage == "contract_fwd":
        return 8.8e3 * n_atoms, "flop"
    if stage == "contract_bwd":
        return 2.8e4 * n_atoms, "flop"
    if stage == "nl_bin":
        # positions and species in; wrapped copies, image counts, cell ids, structure ids,
        # the cell-ordered atom list and the sorted float4 copies out
        return (28.0 + 48.0 + 8.0 + 44.0) * n_atoms, "byte"
    if stage == "nl_count":
        return (16.0 + 4.0) * n_atoms, "byte"
    if stage == "nl_scan":
        return 8.0 * n_atoms, "byte"
    if stage == "nl_fill":
        return 16.0 * n_atoms + 4.0 * n_atoms + 8.0 * n_pairs, "byte"
    if stage in ("nl_coop", "neighbors"):
        # what the build must move: positions in (24 B), sorted coordinates out (24 B),
        # permutation / cell index (8 B) per atom; column index (4 B) and image shift (3 B)
        # per pair
        return NL_BYTES_PER_ATOM * n_atoms + NL_BYTES_PER_PAIR * n_pairs, "byte"
    if stage == "reduce":
        # output-layer partials (H / 32 per atom) and the species index in
        return 4.0 * n_atoms * (H // 32 + 1), "byte"
    return 0.0, "flop"


# source files whose kernels each stage runs (a traffic figure is void once they change)
STAGE_SOURCES = {
    "nl_coop": ("gm_nlist.cu",), "neighbors": ("gm_nlist.cu",), "moments": ("gm_pair.cu", "gm_common.cuh"),
    "forces": ("gm_pair.cu", "gm_common.cuh"), "contract_fwd": ("gm_contract.cu",),
    "contract_bwd": ("gm_contract.cu",), "mlp_fused": ("gm_mlp_fused.cuh", "gm_mlp_cluster.cuh", "gm_gemm_tc.cuh"),
}
# the network GEMM stages run the tensor-core kernel (mixed) or the FFMA kernel (FP32)
STAGE_SOURCES.update({g: ("gm_gemm.h", "gm_gemm_tc.cuh", "gm_gemm_tc.cu", "gm_gemm_simt.cu")
                      for g in ("gemm_l1", "gemm_l2", "gemm_b1", "gemm_b0")})

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture
# of the stage's kernel on the named workload and precision, with the hash of its sources at
# that time (the capture commands and figures are under profiles/).  "scaled": captured on a
# smaller crystal of the same density and scaled by its atom (and pair) count.
TRAFFIC = {
    ("nl_coop", WORKLOADS[2], "mixed"): {"bytes_per_launch": 150784, "source_sha16": "705382e9780d2994",
                                         "capture": "profiles/nl_coop_emim1536.md"},
    ("gemm_l2", WORKLOADS[2], "fp32"): {"bytes_per_launch": 4241920, "source_sha16": "e58e72bb40f7f696",
                                        "capture": "profiles/traffic_dominant_kernels.md"},
    ("nl_coop", WORKLOADS[3], "mixed"): {"bytes_per_launch": 9254144, "source_sha16": "705382e9780d2994",
                                         "capture": "profiles/traffic_dominant_kernels.md"},
    ("gemm_b0", WORKLOADS[3], "fp32"): {"bytes_per_launch": 128016896, "source_sha16": "e58e72bb40f7f696",
                                        "capture": "profiles/traffic_dominant_kernels.md"},
    ("forces", WORKLOADS[5], "mixed"): {"bytes_per_launch": 2 * 73158400, "source_sha16": "4e689b987fa8f6c8",
                                        "capture": "profiles/traffic_dominant_kernels.md (65,536 atoms, scaled x2)"},
    ("gemm_l2", WORKLOADS[5], "fp32"): {"bytes_per_launch": 2 * 236163328, "source_sha16": "e58e72bb40f7f696",
                                        "capture": "profiles/traffic_dominant_kernels.md (65,536 atoms, scaled x2)"},
}


def max_over_ranks(x):
    """The largest x over the ranks of the process group (x itself when there is none): a job of
    independent replicas takes as long as its slowest one."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _world():
    return int(os.environ.get("WORLD_SIZE", "1"))


def replica_throughput(n_atoms, steps, seconds, world):
    """Whole-job atom-steps/s of `world` independent replicas of an n_atoms-atom system, each
    running `steps` steps, the job taking `seconds` (its slowest replica's time)."""
    return world * n_atoms * steps / seconds


def source_sha16(stage):
    import hashlib
    h = hashlib.sha256()
    for f in STAGE_SOURCES.get(stage, ()):
        h.update((ROOT / "paper_2505_22168_b300" / "csrc" / f).read_bytes())
    return h.hexdigest()[:16]


def traffic_for(stage, workload, precision):
    """(bytes per launch, capture) of the stage on the workload, or (None, None) when there is no
    capture or the stage's sources changed since it was taken."""
    t = TRAFFIC.get((stage, workload, precision))
    if t is None or t["source_sha16"] != source_sha16(stage):
        return None, None
    return t["bytes_per_launch"], t["capture"]


def measure_alu_peaks():
    """FP32 FMA and special-function-unit (ex2) throughput of this GPU, measured with the
    library's probe kernels (gm_probe_alu): best of five timed launches after one warm-up."""
    import torch

    from paper_2505_22168_b300 import _lib
    from paper_2505_22168_b300.gmnn import _ptr, _stream
    sink = torch.zeros(8192, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    out = {}
    for kind, name, iters, scale in ((0, "fp32_fma_tflops", 16384, 1e12), (1, "mufu_ex2_gops", 2048, 1e9)):
        best = 0.0
        for rep in range(6):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ops = _lib.gm_probe_alu(kind, iters, _ptr(sink), _stream())
            e1.record(stream)
            e1.synchronize()
            if rep > 0:
                best = max(best, ops / (e0.elapsed_time(e1) * 1e-3))
        out[name] = round(best / scale, 2)
    out["how"] = "gm_probe_alu: independent FMA / ex2.approx chains on every SM, CUDA events, best of 5"
    return out


def roofline(stages, n_atoms, n_pairs, H, precision, peaks, sustained, workload=None):
    busy = {k: v for k, v in stages.items() if v[1] > 0}
    if any(k.startswith("nl_") for k in busy):
        busy.pop("neighbors", None)   # its sub-stages are timed on their own
    if not busy:
        return None, {}
    per = {k: v[0] / v[1] for k, v in busy.items()}
    total = sum(v[0] for v in busy.values())
    share = {k: round(v[0] / total, 4) for k, v in busy.items()}
    top = max(per, key=lambda k: busy[k][0])
    work, unit = algorithmic_work(top, n_atoms, n_pairs, H)
    sec = per[top] / 1e3
    if unit == "byte":
        achieved = work / sec / 1e9
        peak = peaks.get("hbm_gbs", 6400.0)
        out = {"bound": "hbm", "unit": "GB/s", "peak_source": "measured hbm_gbs" if "hbm_gbs" in peaks else "fallback"}
    elif (top.startswith("gemm") or top == "mlp_fused") and precision == "mixed":
        achieved = work / sec / 1e12
        key = "bf16_tflops_sustained" if sustained else "bf16_tflops"
        peak = peaks.get(key, 1400.0 if sustained else 1800.0)
        out = {"bound": "tensor", "unit": "TFLOP/s", "peak_source": f"measured {key}" if key in peaks else "fallback"}
    else:
        achieved = work / sec / 1e12
        if "fp32_fma_tflops" in peaks:
            peak = peaks["fp32_fma_tflops"]
            src = "measured fp32_fma_tflops (gm_probe_alu, this run)"
        else:
            peak = FP32_ALU_PEAK_TFLOPS
            src = "derived: 148 SMs x 128 FP32 FMA/clk x 2 flop x 2032 MHz"
        out = {"bound": "alu", "unit": "TFLOP/s", "peak_source": src}
    traffic, capture = traffic_for(top, workload, precision)
    out.update({"kernel": top, "achieved": round(achieved, 3), "peak": round(peak, 2),
                "frac": round(achieved / peak, 4), "traffic": traffic, "traffic_capture": capture,
                "ms_per_launch": round(per[top], 5), "algorithmic_work_per_launch": work, "work_unit": unit})
    return out, share


# ----------------------------------------------------------------------------- GPU arm

def run_gpu(args, cfg, precision, steps, warmup, world, rank, measure_e2e, clock_sampler=None,
            measure_accuracy=False):
    import torch

    import synth
    from paper_2505_22168_b300 import GMNN, DeviceSystem, _lib

    batch, desc, params = synth.config(cfg)
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    model = GMNN(desc, params, precision=precision)
    sysd = DeviceSystem(batch)
    nl = model.build_neighbors(sysd)
    path = jitter_path(batch, 7000 + cfg, warmup + max(steps, E2E_STEPS)) if cfg == 2 else None
    n = batch.n_atoms
    if path is not None:
        pos_dev = [torch.as_tensor(path[k], device=model.device) for k in range(warmup + steps)]
    else:
        pos_dev = [sysd.pos] * (warmup + steps)
    # capacity with headroom for the jitter (checked after the run)
    cap = int(nl.capacity * 1.05) + 1024
    from paper_2505_22168_b300 import NeighborList
    nl = NeighborList(n, cap, model.device)
    out = (torch.empty(batch.n_structures, dtype=torch.float64, device=model.device),
           torch.empty(n, 3, dtype=torch.float32, device=model.device), None)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=model.device)
    stream = torch.cuda.current_stream()

    # the steps read their positions where they are resident (a device buffer per step); the
    # warm-up, the tuning and the stage timing copy them into one buffer, pos_buf
    pos_buf = torch.empty_like(sysd.pos)
    sysd.pos = pos_buf
    tuning = None
    if args.tune:
        # launch shapes picked by timing graph replays (untimed set-up; results are identical
        # for every setting)
        from paper_2505_22168_b300 import autotune
        pos_buf.copy_(pos_dev[0])
        reps = 10 if n > 50000 else 20

        def flushed_timer(m):
            # the quantity the bench reports: one replay between events after an L2 flush
            g = m.capture_step(sysd, nl, out)
            g.replay()
            e = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            for e0, e1 in e:
                flush.zero_()
                e0.record(stream)
                g.replay()
                e1.record(stream)
            stream.synchronize()
            if m.read_status() != 0:
                raise RuntimeError(f"device status {m.read_status()} while tuning")
            del g
            return float(np.median([e0.elapsed_time(e1) for e0, e1 in e]))

        t = autotune.tune(model, sysd, nl, out, reps=reps, timer=flushed_timer)
        tuning = {"settings": t["settings"], "tuned_ms": round(t["ms"], 5), "default_ms": round(t["default_ms"], 5),
                  "trials": len(t.get("trials", [])), "timed_as": "median of single replays after an L2 flush"}

    def step(k):                       # stream launches
        pos_buf.copy_(pos_dev[k])
        model.step(sysd, nl, out)

    for k in range(warmup):
        step(k)
    stream.synchronize()
    if model.read_status() != 0:
        raise RuntimeError(f"device status {model.read_status()} during warm-up")
    n_pairs = int(nl.n_pairs.item())

    # per-step launch count (library kernels), measured on one uncaptured step
    _lib.gm_profile_reset()
    step(0)
    stream.synchronize()
    per_step_launches = _lib.gm_profile_collect()[1]

    # one graph per timed step, captured on that step's resident positions (untimed set-up): a
    # timed step is the library's launches alone, with no copy into a shared input buffer
    graphs = []
    if args.graph:
        for k in range(steps):
            sysd.pos = pos_dev[warmup + k]
            graphs.append(model.capture_step(sysd, nl, out))
        sysd.pos = pos_buf

    def timed(k, use_graph):
        flush.zero_()
        if use_graph:
            ev0[k].record(stream)
            graphs[k].replay()
        else:
            sysd.pos = pos_dev[warmup + k]
            ev0[k].record(stream)
            model.step(sysd, nl, out)
            sysd.pos = pos_buf
        ev1[k].record(stream)

    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    stream.synchronize()
    if clock_sampler is not None:
        clock_sampler.__enter__()
    for k in range(steps):
        timed(k, bool(graphs))
    stream.synchronize()
    if clock_sampler is not None:
        clock_sampler.__exit__(None, None, None)
    status = model.read_status()
    if status != 0:
        raise RuntimeError(f"device status {_lib.STATUS_NAMES.get(status, status)} in the timed region")
    ms = sum(ev0[k].elapsed_time(ev1[k]) for k in range(steps))
    launches = per_step_launches * steps
    # stage timing: a second pass over the same steps with the library's stage events; in
    # graph mode a second graph is captured with the events as record nodes and read after
    # every replay, so the stage times carry no host launch gaps
    stages, ms_stream = {}, float("nan")
    if args.stage_timing:
        _lib.gm_profile_enable(True)
        gprof = model.capture_step(sysd, nl, out) if graphs else None
        _lib.gm_profile_reset()
        for k in range(steps):
            flush.zero_()
            ev0[k].record(stream)
            pos_buf.copy_(pos_dev[warmup + k])
            if gprof is not None:
                gprof.replay()
            else:
                model.step(sysd, nl, out)
            ev1[k].record(stream)
            if gprof is not None:          # read this replay's record nodes
                stream.synchronize()
                stages, _ = _lib.gm_profile_collect()
        stream.synchronize()
        _lib.gm_profile_enable(False)
        if gprof is None:
            stages, _ = _lib.gm_profile_collect()
        _lib.gm_profile_forget_graphs()
        del gprof
        ms_stream = sum(ev0[k].elapsed_time(ev1[k]) for k in range(steps))
    ms = max_over_ranks(ms)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    # device memory of the step: torch's peak (inputs, outputs, neighbour list, workspaces, the
    # captured graphs' pools) without the benchmark's own buffers, plus the model's weights
    bench_bytes = FLUSH_BYTES + (len(pos_dev) * sysd.pos.numel() * 8 if path is not None else 0)
    peak_torch = torch.cuda.max_memory_allocated()
    memory = {"peak_bytes": int(peak_torch - bench_bytes + _lib.gm_model_device_bytes(model.handle)),
              "torch_max_allocated_bytes": int(peak_torch), "benchmark_buffers_bytes": int(bench_bytes),
              "model_weights_bytes": int(_lib.gm_model_device_bytes(model.handle)),
              "workspace_bytes": {"neighbors": int(model.workspace(_lib.GM_OP_NEIGHBORS, sysd, nl.capacity)[1]),
                                  "energy_forces": int(model.workspace(_lib.GM_OP_ENERGY_FORCES, sysd, nl.capacity)[1])},
              "neighbour_list_bytes": int(nl.capacity * 8 + (n + 1) * 4)}
    accuracy = None
    if measure_accuracy and cfg == 3:
        accuracy = batch_accuracy(batch, desc, params, out[0].cpu().numpy(), out[1].cpu().numpy(), range(0, 256, 16))
    elif measure_accuracy and cfg == 5:
        accuracy = sampled_accuracy(batch, desc, params, out[1].cpu().numpy(), 12)
    res = {"ms_total": ms, "ms_per_step": ms / steps, "n_atoms": n, "n_pairs": n_pairs, "stages": stages,
           "memory": memory, "accuracy": accuracy,
           "launches": launches, "H": desc["n_hidden"], "value": replica_throughput(n, steps, ms / 1e3, world),
           "launch_mode": "cuda-graph replay" if graphs else "stream launches", "tuning": tuning,
           "ms_per_step_stream_with_stage_events": ms_stream / steps}

    if measure_e2e:
        # end to end through the public API with host buffers: pinned positions in,
        # energies and forces out, copies inside the timed region
        e2e_steps = E2E_STEPS
        host_pos = [torch.as_tensor(path[warmup + k] if path is not None else batch.pos).pin_memory()
                    for k in range(e2e_steps)]
        # graph mode: one graph per in-flight slot holding the copy of the slot's pinned input
        # positions to the device, the step, and the copies of energies and forces back to the
        # slot's pinned host buffers.  Two steps are in flight: the host writes step k's
        # positions into a free slot and replays its graph while the GPU still runs step k - 1,
        # then waits for step k - 1 and reads its energies and forces (the steps are
        # independent evaluations; the device buffers are shared and the stream orders them)
        slots = 2 if graphs else 1
        E_host = [torch.empty(batch.n_structures, dtype=torch.float64).pin_memory() for _ in range(slots)]
        F_host = [torch.empty(n, 3, dtype=torch.float32).pin_memory() for _ in range(slots)]
        pin_in = [torch.empty_like(host_pos[0]).pin_memory() for _ in range(slots)]
        g_e2e = []
        if graphs:
            for sl in range(slots):
                pin_in[sl].copy_(host_pos[0])
                torch.cuda.synchronize()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g):
                    pos_buf.copy_(pin_in[sl], non_blocking=True)
                    model.step(sysd, nl, out)
                    E_host[sl].copy_(out[0], non_blocking=True)
                    F_host[sl].copy_(out[1], non_blocking=True)
                g.replay()
                g_e2e.append(g)
        torch.cuda.synchronize()
        pin_np = [t.numpy() for t in pin_in]          # the pinned inputs as the host program sees them
        E_np = [t.numpy() for t in E_host]
        F_np = [t.numpy() for t in F_host]
        host_np = [h.numpy() for h in host_pos]
        done = [torch.cuda.Event() for _ in range(slots)]
        checksum = 0.0
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        t0 = time.perf_counter()
        for k in range(e2e_steps + slots - 1):
            sl = k % slots
            if k >= slots:                           # step k - slots: wait, read its results
                done[sl].synchronize()
                checksum += float(E_np[sl][0]) + float(F_np[sl][0, 0])
            if k >= e2e_steps:
                continue
            if g_e2e:
                np.copyto(pin_np[sl], host_np[k])
                g_e2e[sl].replay()
            else:
                pos_buf.copy_(host_pos[k], non_blocking=True)
                model.step(sysd, nl, out)
                E_host[sl].copy_(out[0], non_blocking=True)
                F_host[sl].copy_(out[1], non_blocking=True)
            done[sl].record(stream)
            if slots == 1:
                done[sl].synchronize()
                checksum += float(E_np[sl][0]) + float(F_np[sl][0, 0])
        wall = max_over_ranks(time.perf_counter() - t0)
        if model.read_status() != 0:
            raise RuntimeError("device status set during the end-to-end run")
        if not np.isfinite(checksum):
            raise RuntimeError("non-finite energies or forces in the end-to-end run")
        res["e2e"] = {"value": replica_throughput(n, e2e_steps, wall, world), "unit": UNIT,
                      "h2d_bytes_per_step": int(host_pos[0].numel() * 8),
                      "d2h_bytes_per_step": int(E_host[0].numel() * 8 + F_host[0].numel() * 4), "steps": e2e_steps,
                      "steps_in_flight": slots}
    del pos_dev, flush
    return res


def run_train(args, steps, warmup, precision="fp32"):
    """Training step on 32 EMIM+BF4- boxes of 96-384 atoms (MLP 2x128): neighbour
    rebuild, energies and forces, force-matching loss against teacher labels, and the
    parameter gradient.  Reference labels come from the FP64 oracle with the teacher's
    parameters (set-up, untimed)."""
    import torch

    import oracle
    import synth
    from synth.configs import teacher_params
    from paper_2505_22168_b300 import GMNN, DeviceSystem, _lib

    batch, desc, params = synth.config(4)
    onl = oracle.neighbors(batch, desc["r_cut"])
    teach = oracle.energy_forces(batch, desc, teacher_params(4), onl, virial=False)
    model = GMNN(desc, params, precision=precision)
    sysd = DeviceSystem(batch)
    nl = model.build_neighbors(sysd)
    from paper_2505_22168_b300 import NeighborList
    nl = NeighborList(batch.n_atoms, int(nl.capacity * 1.05) + 1024, model.device)
    Eref = torch.as_tensor(teach["E"], device=model.device)
    Fref = torch.as_tensor(teach["F"], dtype=torch.float32, device=model.device)
    stream = torch.cuda.current_stream()
    out = (torch.empty(batch.n_structures, dtype=torch.float64, device=model.device),
           torch.empty(batch.n_atoms, 3, dtype=torch.float32, device=model.device), None)

    last = {}

    def step():
        model.clear_status()
        model.build_neighbors(sysd, nl, check=False)
        model.energy_forces(sysd, nl, out=out, clear=False)
        loss, gE, gF = model.force_matching_loss(sysd, out[0], Eref, out[1], Fref)
        last["loss"] = loss
        last["grad"] = model.param_grad(sysd, nl, gE, gF, clear=False)
        return last["grad"]

    for _ in range(warmup):
        step()
    stream.synchronize()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    _lib.gm_profile_reset()
    _lib.gm_profile_enable(args.stage_timing)
    for k in range(steps):
        ev0[k].record(stream)
        step()
        ev1[k].record(stream)
    stream.synchronize()
    _lib.gm_profile_enable(False)
    stages, launches = _lib.gm_profile_collect()
    if model.read_status() != 0:
        raise RuntimeError("device status set in the training run")
    ms = sum(ev0[k].elapsed_time(ev1[k]) for k in range(steps))
    if any(k.startswith("nl_") and v[1] > 0 for k, v in stages.items()):
        stages = {k: v for k, v in stages.items() if k != "neighbors"}
    total = sum(v[0] for v in stages.values() if v[1] > 0) or 1.0
    # accuracy of the whole training step: the oracle's loss and parameter gradient at the same
    # parameters and labels (FP64 energies and forces, then the hand-derived gradient)
    from paper_2505_22168_b300 import unpack_theta
    ref = oracle.energy_forces(batch, desc, params, onl, virial=False)
    L_o, gE_o, gF_o = oracle.loss(batch, ref["E"], teach["E"], ref["F"], teach["F"].astype(np.float32).astype(np.float64))
    go = oracle.param_grad(batch, desc, params, onl, gE_o, gF_o)
    g = unpack_theta(last["grad"].cpu().numpy().astype(np.float64), desc["n_species"], desc["n_hidden"])
    rel = {k: float(np.linalg.norm(g[k].ravel() - go[k].ravel()) / np.linalg.norm(go[k].ravel())) for k in go}
    accuracy = {"loss": float(abs(float(last["loss"].item()) - L_o) / abs(L_o)),
                "param_grad_rel_l2_worst_group": max(rel.values()),
                "param_grad_worst_group": max(rel, key=rel.get),
                "reference": "FP64 oracle loss and parameter gradient on the same batch, parameters and labels"}
    ms = max_over_ranks(ms)
    return {"workload": "emim-train-32 (32 EMIM+BF4- boxes, 7920 atoms, r_cut 5 A, MLP 2x128)",
            "accuracy": accuracy,
            "precision": precision, "step": "neighbours + energy/forces + loss + parameter gradient",
            "value": replica_throughput(batch.n_atoms, steps, ms / 1e3, _world()), "unit": UNIT,
            "ms_per_step": ms / steps,
            "steps": steps, "stage_share": {k: round(v[0] / total, 4) for k, v in stages.items() if v[1] > 0}}


def md_system(n_atoms):
    """The paper's Li3PO4 MD sizes (Table li3po4_perf): a 192-atom box and its 3x3x3 supercell of
    5184 atoms (synthetic jittered crystal, 2.4 g/cm^3), the batch workload's model (r_cut 5 A,
    MLP 2x256), Maxwell-Boltzmann velocities at 600 K."""
    import synth
    from synth.params import maxwell_boltzmann
    from synth.systems import li3po4_crystal, make_batch, species_masses, supercell
    _, desc, params = synth.config(3)
    base = li3po4_crystal(24, 4242, sigma=0.05)
    s = base if n_atoms == 192 else supercell(base, 3)
    b = make_batch([s], 3)
    masses = species_masses("li3po4")
    vel = maxwell_boltzmann(masses[b.species], b.atom_ptr, 600.0, 4242)
    return b, desc, params, masses, vel


def run_md(args, n_atoms, precision, n_inner=100, replays=5):
    """Whole MD steps on the device (section "Deployment"; the appendix's configuration: NVT at
    600 K, 0.5 fs, Nose-Hoover chain 3/2/3, tau 100 steps, skin 0.5 A): half kick, drift, skin
    test, neighbour rebuild when needed, energies and forces, half kick, thermostat.  A CUDA
    graph of n_inner steps is replayed; each replay is timed with CUDA events (L2 not flushed:
    the state of an MD run stays resident between steps, which is the workload)."""
    import torch

    from paper_2505_22168_b300 import GMNN, DeviceSystem, MDParams, MDState, _lib
    b, desc, params, masses, vel = md_system(n_atoms)
    m = GMNN(desc, params, precision=precision)
    sysd = DeviceSystem(b)
    mp = MDParams(dt=0.5, skin=0.5, temperature=600.0, ensemble="nvt")
    nl = m.md_neighbor_list(sysd, mp)
    st = MDState(sysd, masses, vel)
    m.md_init(sysd, nl, mp, st)
    g = m.capture_md(sysd, nl, mp, st, n_inner)
    for _ in range(max(1, args.warmup // 2)):
        g.replay()
    stream = torch.cuda.current_stream()
    stream.synchronize()
    b0 = int(st.n_builds.item())
    _lib.gm_profile_reset()
    m.md_run(sysd, nl, mp, st, 1)                 # one uncaptured step: launches per step
    stream.synchronize()
    launches_per_step = _lib.gm_profile_collect()[1]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(replays)]
    for e0, e1 in ev:
        e0.record(stream)
        g.replay()
        e1.record(stream)
    stream.synchronize()
    if m.read_status() != 0:
        raise RuntimeError(f"device status {m.read_status()} in the MD run")
    ms = sum(e0.elapsed_time(e1) for e0, e1 in ev)
    steps = n_inner * replays
    builds = int(st.n_builds.item()) - b0
    ms = max_over_ranks(ms)
    us_atom_step = ms * 1e3 / (steps * n_atoms)
    # accuracy at the final configuration: the forces the integrator used against the oracle's
    import oracle
    pos = st.pos.cpu().numpy()
    F = st.forces.cpu().numpy()
    import dataclasses
    bf = dataclasses.replace(b, pos=pos)
    if n_atoms <= 1000:
        ref = oracle.energy_forces(bf, desc, params, oracle.neighbors(bf, desc["r_cut"]), virial=False)
        acc = _errors(st.energy.cpu().numpy(), F, ref["E"], ref["F"], ref["E_atom"], b.atom_ptr)
        acc["reference"] = "FP64 oracle at the final configuration (full evaluation)"
    else:
        acc = sampled_accuracy(bf, desc, params, F, 12)
    return {"workload": f"li3po4-md-{n_atoms} (Li3PO4-like crystal, {n_atoms} atoms, r_cut 5 A, MLP 2x256, "
                        f"NVT 600 K, dt 0.5 fs, NHC 3/2/3, skin 0.5 A)",
            "precision": precision, "step": "whole MD step (thermostat, Verlet, skin test, rebuilds, E/F)",
            "value": replica_throughput(n_atoms, steps, ms / 1e3, _world()), "unit": UNIT, "ms_per_step": ms / steps,
            "us_per_atom_per_step": us_atom_step, "steps": steps, "n_inner": n_inner,
            "neighbour_builds": builds, "launches_per_step": launches_per_step,
            "launch_mode": "cuda-graph replay of n_inner steps", "accuracy": acc,
            "paper_context": {"us_per_atom_per_step": {"192": 10.1, "5184": 2.3},
                              "hardware": "V100, Apax JAX MD engine (Table li3po4_perf)"}}


# ----------------------------------------------------------------------------- CPU (oracle)

ENS_HEADS = 8


def run_readout_variant(args, kind, precision, steps, warmup, measure_accuracy=True):
    """The headline workload (1536-atom EMIM+BF4- box, r_cut 6 A, MLP 2x512) with the other
    radial basis or readout the library builds: the Bessel-like basis ("bessel"), or a
    shallow ensemble of ENS_HEADS output heads with forces as the gradient of the mean energy
    plus the energy spread ("ensemble-mean"), or also every head's forces and the force
    spread ("ensemble-jacobian").  Step = neighbour rebuild + this evaluation, replayed as one
    CUDA graph, L2 flushed between steps (base positions every step); the errors against the
    FP64 oracle at the same positions."""
    import torch

    import oracle
    import synth
    from synth.configs import emim_number_density, mean_neighbours
    from synth.params import make_params
    from paper_2505_22168_b300 import GMNN, DeviceSystem, NeighborList

    batch, desc, params = synth.config(2)
    if kind == "bessel":
        desc = dict(desc, basis="bessel")
    else:
        desc = dict(desc, n_ensemble=ENS_HEADS)
        pe = make_params(desc["n_species"], desc["n_hidden"], 1202,
                         mean_neighbours(emim_number_density(), desc["r_cut"]), n_ensemble=ENS_HEADS)
        params = dict(params, w3=pe["w3"], b3=pe["b3"])
    model = GMNN(desc, params, precision=precision)
    sysd = DeviceSystem(batch)
    nl = model.build_neighbors(sysd)
    nl = NeighborList(batch.n_atoms, int(nl.capacity * 1.05) + 1024, model.device)
    n = batch.n_atoms
    stream = torch.cuda.current_stream()
    out = (torch.empty(batch.n_structures, dtype=torch.float64, device=model.device),
           torch.empty(n, 3, dtype=torch.float32, device=model.device), None)
    mode = "jacobian" if kind == "ensemble-jacobian" else "mean"
    res = {}

    def step():
        if kind == "bessel":
            model.step(sysd, nl, out)
        else:
            model.clear_status()
            model.build_neighbors(sysd, nl, check=False)
            res["o"] = model.energy_forces_ensemble(sysd, nl, mode=mode)

    for _ in range(warmup):
        step()
    stream.synchronize()
    model.check_status()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    graph.replay()
    stream.synchronize()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=model.device)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for e0, e1 in ev:
        flush.zero_()
        e0.record(stream)
        graph.replay()
        e1.record(stream)
    stream.synchronize()
    model.check_status()
    ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / steps
    accuracy = None
    if measure_accuracy:
        onl = oracle.neighbors(batch, desc["r_cut"])
        ap = np.asarray(batch.atom_ptr)
        if kind == "bessel":
            ref = oracle.energy_forces(batch, desc, params, onl, virial=False)
            accuracy = _errors(out[0].cpu().numpy(), out[1].cpu().numpy(), ref["E"], ref["F"], ref["E_atom"], ap)
        else:
            ref = oracle.energy_forces_ensemble(batch, desc, params, onl, virial=False)
            o = res["o"]
            accuracy = _errors(o["E"].cpu().numpy(), o["F"].cpu().numpy(), ref["E"], ref["F"], ref["E_atom"], ap)
            accuracy["energy_spread_abs"] = float(np.abs(o["E_std"].cpu().numpy() - ref["E_std"]).max())
            accuracy["energy_spread_ref"] = float(np.abs(ref["E_std"]).max())
            if mode == "jacobian":
                Fh = o["F_heads"].cpu().numpy().astype(np.float64)
                accuracy["head_force_rms_worst"] = max(
                    _errors(None, Fh[k], None, ref["F_heads"][k], None, ap)["force_rms"] for k in range(ENS_HEADS))
        accuracy["reference"] = "FP64 oracle at the same positions (full evaluation)"
    del graph, flush
    name = {"bessel": "emim-64pairs-1536-bessel (the headline box with the Bessel-like radial basis)",
            "ensemble-mean": f"emim-64pairs-1536-ensemble{ENS_HEADS}-mean (the headline box, {ENS_HEADS}-head "
                             "shallow ensemble: mean energy, its gradient, energy spread)",
            "ensemble-jacobian": f"emim-64pairs-1536-ensemble{ENS_HEADS}-jacobian (the headline box, {ENS_HEADS}-head "
                                 "shallow ensemble: also every head's forces and the force spread)"}[kind]
    ms = max_over_ranks(ms)
    return {"workload": name, "precision": precision, "value": replica_throughput(n, 1, ms / 1e3, _world()),
            "unit": UNIT, "ms_per_step": ms,
            "steps": steps, "step": "neighbour rebuild + evaluation", "launch_mode": "cuda-graph replay",
            "l2": "256 MiB buffer written between timed steps", "accuracy": accuracy}


def oracle_step_seconds(cfg, budget_s, max_evals=None, keep=False):
    """Time the FP64 oracle (brute-force neighbours + energy/forces) on the workload's
    structure; repeats until budget_s of CPU time or max_evals evaluations.  With keep, also
    returns the last evaluation's result."""
    import oracle
    import synth

    batch, desc, params = synth.config(cfg)
    oracle.build()
    times = []
    ref = None
    t_start = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        nl = oracle.neighbors(batch, desc["r_cut"])
        ref = oracle.energy_forces(batch, desc, params, nl, virial=True)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start >= budget_s or (max_evals and len(times) >= max_evals):
            break
    if keep:
        return batch.n_atoms, times, oracle.num_threads(), ref
    return batch.n_atoms, times, oracle.num_threads()


def accuracy_vs_oracle(cfg, ref):
    """Errors of both GPU paths against the oracle's result for the same positions (the
    metrics of the parity tests: energy per atom relative to the rms atomic energy, force
    RMS and largest element relative to the rms reference force)."""
    import torch

    import synth
    from paper_2505_22168_b300 import GMNN, DeviceSystem

    batch, desc, params = synth.config(cfg)
    out = {"reference": "FP64 oracle at the workload's base positions"}
    for prec in ("fp32", "mixed"):
        if prec == "mixed" and not _mixed_available():
            continue
        m = GMNN(desc, params, precision=prec)
        sysd = DeviceSystem(batch)
        nl = m.build_neighbors(sysd)
        E, F, _ = m.energy_forces(sysd, nl)
        m.check_status()
        E = E.cpu().numpy()
        F = F.cpu().numpy().astype(np.float64)
        ap = batch.atom_ptr
        e_err = max(abs(E[b] - ref["E"][b]) / (ap[b + 1] - ap[b]) / np.sqrt((ref["E_atom"][ap[b]:ap[b + 1]] ** 2).mean())
                    for b in range(batch.n_structures) if ap[b + 1] > ap[b])
        rms = np.sqrt((ref["F"] ** 2).mean())
        dF = F - ref["F"]
        out[prec] = {"energy": float(e_err), "force_rms": float(np.sqrt((dF ** 2).mean()) / rms),
                     "force_max": float(np.abs(dF).max() / rms)}
        del m
        torch.cuda.synchronize()
    return out


def _errors(E, F, Eref, Fref, E_atom_ref, atom_ptr):
    """Parity metrics: energy per atom over the rms atomic energy (worst structure), force
    RMS and largest element over the rms reference force."""
    out = {}
    if E is not None:
        e = 0.0
        for b in range(len(atom_ptr) - 1):
            a0, a1 = atom_ptr[b], atom_ptr[b + 1]
            if a1 > a0:
                e = max(e, abs(E[b] - Eref[b]) / (a1 - a0) / np.sqrt((E_atom_ref[a0:a1] ** 2).mean()))
        out["energy"] = float(e)
    rms = np.sqrt((Fref ** 2).mean())
    dF = F.astype(np.float64) - Fref
    out["force_rms"] = float(np.sqrt((dF ** 2).mean()) / rms)
    out["force_max"] = float(np.abs(dF).max() / rms)
    return out


def batch_accuracy(batch, desc, params, E, F, idx):
    """Errors of a batched run on a subset of its structures, against the FP64 oracle on those
    structures alone (structures are independent, so this is exact for them)."""
    import oracle
    from synth.systems import make_batch
    idx = list(idx)
    ap = batch.atom_ptr
    sub = make_batch([(batch.pos[ap[b]:ap[b + 1]], batch.species[ap[b]:ap[b + 1]], batch.cell[b]) for b in idx],
                     batch.n_species)
    ref = oracle.energy_forces(sub, desc, params, oracle.neighbors(sub, desc["r_cut"]), virial=False)
    rows = np.concatenate([np.arange(ap[b], ap[b + 1]) for b in idx])
    out = _errors(E[idx], F[rows], ref["E"], ref["F"], ref["E_atom"], sub.atom_ptr)
    out["reference"] = f"FP64 oracle on {len(idx)} of the {batch.n_structures} structures ({sub.n_atoms} atoms)"
    return out


def sampled_accuracy(batch, desc, params, F, n_rows):
    """Force errors of a large system on sampled atoms, against an exact oracle evaluation of
    those atoms (oracle.sampled_forces)."""
    import oracle
    rows = np.sort(np.random.default_rng(31).choice(batch.n_atoms, n_rows, replace=False))
    ref = oracle.sampled_forces(batch, desc, params, rows)
    out = _errors(None, F[ref["rows"]], None, ref["F"], None, None)
    out["reference"] = (f"FP64 oracle forces of {n_rows} sampled atoms (exact sub-evaluation over "
                        f"{ref['n_sub_atoms']} atoms); energies not compared at this size")
    return out


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def cpu_baseline(cfg, budget_s):
    """The oracle on all host threads (budget_s), then on one thread (a quarter of that)."""
    import oracle
    n, times, threads, ref = oracle_step_seconds(cfg, budget_s, keep=True)
    value = n * len(times) / sum(times)
    oracle.set_threads(1)
    try:
        _, t1, _ = oracle_step_seconds(cfg, budget_s / 4)
    finally:
        oracle.set_threads(threads)
    return {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{len(times)} full evaluations (brute-force neighbours + E/F/virial, FP64) of the "
                      f"{n}-atom workload, {sum(times):.1f} s on {threads} OpenMP threads",
            "value_1core": n * len(t1) / sum(t1),
            "sample_1core": f"{len(t1)} full evaluations, {sum(t1):.1f} s on 1 thread",
            "cpu_model": cpu_model(), "nproc": os.cpu_count()}, ref


# ----------------------------------------------------------------------------- main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["auto", "fp32", "mixed"], default="auto")
    ap.add_argument("--config", type=int, choices=[2, 3, 5], default=2)
    ap.add_argument("--tune", type=int, default=1, help="autotune launch shapes before timing")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the oracle checks of the variants")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--stage-timing", type=int, default=1)
    ap.add_argument("--graph", type=int, default=1, help="replay the step as a CUDA graph")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        n, times, threads = oracle_step_seconds(args.config, budget_s=1e9, max_evals=args.warmup + args.steps)
        timed = times[args.warmup:] if len(times) > args.warmup else times
        value = n * len(timed) / sum(timed)
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                "steps": len(timed), "warmup": args.warmup, "ms_per_step": 1e3 * sum(timed) / len(timed),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": WORKLOADS[args.config], "path": "FP64 CPU oracle (plain C + OpenMP)"},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                                 "sample": f"{len(timed)} timed full evaluations of the {n}-atom workload"},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    else:
        torch.cuda.set_device(0)

    from paper_2505_22168_b300 import build
    build.build()
    precision = args.precision
    if precision == "auto":
        precision = "mixed" if _mixed_available() else "fp32"

    peaks = {}
    pk = ROOT / "MEASURED_PEAKS.json"
    if pk.exists():
        peaks = json.loads(pk.read_text())

    alu_peaks = measure_alu_peaks()
    peaks = dict(peaks, **{k: v for k, v in alu_peaks.items() if k != "how"})
    sampler = ClockSampler(local_rank)
    head = run_gpu(args, args.config, precision, args.steps, args.warmup, world, rank, True, sampler)
    clocks = sampler.summary()
    roof, share = roofline(head["stages"], head["n_atoms"], head["n_pairs"], head["H"], precision, peaks,
                           sustained=False, workload=WORKLOADS[args.config])

    # errors of both paths at the headline workload's base positions (the oracle run doubles
    # as the CPU baseline's sample)
    cpu = None
    accuracy = None
    accuracy_by_prec = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, ref = cpu_baseline(args.config, args.cpu_seconds)
        accuracy = accuracy_vs_oracle(args.config, ref)
        accuracy_by_prec = {k: v for k, v in accuracy.items() if k in ("fp32", "mixed")}

    variants = []
    if not args.no_variants:
        for cfg in (2, 3, 5):
            for prec in ("fp32", "mixed"):
                if (cfg, prec) == (args.config, precision):
                    continue
                if prec == "mixed" and not _mixed_available():
                    continue
                steps = max(5, args.steps // {2: 1, 3: 2, 5: 5}[cfg])
                r = run_gpu(args, cfg, prec, steps, args.warmup, world, rank, False,
                            measure_accuracy=rank == 0 and not args.no_accuracy)
                rf, sh = roofline(r["stages"], r["n_atoms"], r["n_pairs"], r["H"], prec, peaks, sustained=False,
                                  workload=WORKLOADS[cfg])
                v = {"workload": WORKLOADS[cfg], "precision": prec, "value": r["value"], "unit": UNIT,
                     "ms_per_step": r["ms_per_step"], "steps": steps, "n_pairs": r["n_pairs"],
                     "launch_mode": r["launch_mode"], "tuning": r["tuning"],
                     "dominant": rf["kernel"] if rf else None, "roofline_frac": rf["frac"] if rf else None,
                     "roofline": rf, "stage_share": sh, "memory": r["memory"], "accuracy": r["accuracy"]}
                if cfg == 2 and accuracy_by_prec is not None:
                    v["accuracy"] = accuracy_by_prec.get(prec)
                variants.append(v)

    if not args.no_variants:
        for prec in ("fp32", "mixed"):
            if prec == "mixed" and not _mixed_available():
                continue
            variants.append(run_train(args, max(5, args.steps // 5), args.warmup, prec))
        for n_md in (192, 5184):
            for prec in ("fp32", "mixed"):
                if prec == "mixed" and not _mixed_available():
                    continue
                variants.append(run_md(args, n_md, prec))
        # the Bessel-like basis and the shallow-ensemble readout on the headline box
        for kind in ("bessel", "ensemble-mean", "ensemble-jacobian"):
            for prec in ("fp32", "mixed"):
                if prec == "mixed" and not _mixed_available():
                    continue
                variants.append(run_readout_variant(args, kind, prec, max(5, args.steps // 2), args.warmup,
                                                    measure_accuracy=rank == 0 and not args.no_accuracy))

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16+f32" if precision == "mixed" else "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.config], "precision": precision, "n_atoms": head["n_atoms"],
                   "n_pairs": head["n_pairs"], "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "256 MiB buffer written between timed steps (outside the step events)",
                   "neighbour_rebuild": "every step", "launch_mode": head["launch_mode"], "tuning": head["tuning"],
                   "stage_timing": "library stage events on a second pass of the same steps "
                                   + ("(a second graph with event-record nodes, "
                                      if head["launch_mode"] == "cuda-graph replay" else "(stream launches, ")
                                   + f"{head['ms_per_step_stream_with_stage_events']:.4f} ms/step)"},
        "roofline": roof, "stage_share": share, "cpu_baseline": cpu, "accuracy": accuracy, "e2e": head.get("e2e"),
        "gpu_launches": head["launches"], "clocks": clocks, "memory": head["memory"], "alu_peaks": alu_peaks,
        "variants": variants,
    }
    print_summary(line)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _short(x):
    return "-" if x is None else f"{x:.2e}"


def print_summary(line):
    """One short line per measured workload on stderr (the JSON line on stdout has it all)."""
    acc = line.get("accuracy") or {}
    rows = [("headline", line["config"]["workload"].split(" ")[0], line["config"]["precision"], line["value"],
             line["ms_per_step"], acc.get(line["config"]["precision"]), (line.get("roofline") or {}).get("frac"),
             (line.get("memory") or {}).get("peak_bytes"))]
    for v in line.get("variants", []):
        rows.append(("variant", v["workload"].split(" ")[0], v.get("precision"), v["value"], v["ms_per_step"],
                     v.get("accuracy"), v.get("roofline_frac"), (v.get("memory") or {}).get("peak_bytes")))
        if "us_per_atom_per_step" in v:
            log(f"         {v['workload'].split(' ')[0]} {v['precision']}: {v['us_per_atom_per_step']:.4f} us/atom/step, "
                f"{v['neighbour_builds']} builds in {v['steps']} steps (paper, V100: "
                f"{v['paper_context']['us_per_atom_per_step']})")
    for kind, wl, prec, val, ms, a, frac, mem in rows:
        a = a or {}
        err = a.get("force_rms", a.get("param_grad_rel_l2_worst_group"))
        log(f"{kind:8s} {wl:22s} {prec:5s} {val / 1e6:8.2f} M atom-steps/s {ms:8.4f} ms  "
            f"F/grad err {_short(err)}  E err {_short(a.get('energy'))}  roof {frac}  "
            f"mem {'-' if mem is None else f'{mem / 2**20:.0f} MiB'}")


def _mixed_available():
    try:
        from paper_2505_22168_b300 import _lib
        return bool(getattr(_lib, "MIXED_AVAILABLE", False))
    except Exception:
        return False


if __name__ == "__main__":
    main()
