"""Small runnable cases of the library's operations, for profilers and quick checks.

    python -m paper_2505_22168_b300.cases neighbors --workload emim1536 --repeat 5
    python -m paper_2505_22168_b300.cases ef --workload li3po4 --units 2048 --precision mixed
    python -m paper_2505_22168_b300.cases param_grad --workload emim-train
    python -m paper_2505_22168_b300.cases md --workload li3po4-md --units 24 --repeat 20

Each case builds its seeded synthetic system, runs the operation once to warm up (buffers,
kernel attributes, tensor maps) and then `--repeat` more times on the current stream, checks
the device status word and prints one line.  Workloads: `emim1536` (64 EMIM+BF4- pairs,
r_cut 6, MLP 2x512), `li3po4` (a jittered Li3PO4-like crystal of `--units` formula units,
8 atoms each, r_cut 6, MLP 2x512), `li3po4-batch` (256 boxes of 32-512 atoms, r_cut 5,
MLP 2x256), `emim-train` (32 EMIM boxes of 96-384 atoms, r_cut 5, MLP 2x128), `li3po4-md` (a
Li3PO4-like crystal of `--units` formula units with the batch model, r_cut 5, MLP 2x256; the
`md` operation runs `--repeat` NVT steps at 600 K, dt 0.5 fs, skin 0.5 A after gm_md_init).
"""
from __future__ import annotations

import argparse
import sys
from pathlib import Path

import torch

sys.path.insert(0, str(Path(__file__).resolve().parent.parent))

import synth  # noqa: E402
from synth.configs import li3po4_number_density, mean_neighbours, model_desc  # noqa: E402
from synth.params import make_params  # noqa: E402
from synth.systems import li3po4_crystal, make_batch  # noqa: E402

from . import GMNN, DeviceSystem  # noqa: E402


def workload(name: str, units: int):
    if name == "emim1536":
        return synth.config(2)
    if name == "li3po4-batch":
        return synth.config(3)
    if name == "emim-train":
        return synth.config(4)
    if name == "li3po4-md":
        b = make_batch([li3po4_crystal(units, 4242, sigma=0.05)], 3)
        _, d, p = synth.config(3)
        return b, d, p
    if name == "li3po4":
        b = make_batch([li3po4_crystal(units, 77, sigma=0.1)], 3)
        d = model_desc(3, 512, 6.0, "silu")
        p = make_params(3, 512, 1005, mean_neighbours(li3po4_number_density(), 6.0))
        return b, d, p
    raise ValueError(f"unknown workload {name!r}")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("op", choices=["neighbors", "ef", "param_grad", "md"])
    ap.add_argument("--workload", default="emim1536")
    ap.add_argument("--units", type=int, default=2048, help="Li3PO4 formula units (8 atoms each)")
    ap.add_argument("--precision", choices=["fp32", "mixed"], default="mixed")
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--tune", action="append", default=[], metavar="KNOB=VALUE",
                    help="library tuning knob, e.g. nl_items=1 (repeatable)")
    args = ap.parse_args(argv)
    torch.cuda.set_device(0)
    b, d, p = workload(args.workload, args.units)
    m = GMNN(d, p, precision=args.precision)
    if args.tune:
        m.set_tuning(**{k: int(v) for k, v in (t.split("=") for t in args.tune)})
    s = DeviceSystem(b)
    if args.op == "md":
        from synth.params import maxwell_boltzmann
        from synth.systems import species_masses
        from . import MDParams, MDState
        masses = species_masses("li3po4")
        mp = MDParams(dt=0.5, skin=0.5, temperature=600.0, ensemble="nvt")
        nl = m.md_neighbor_list(s, mp)
        st = MDState(s, masses, maxwell_boltzmann(masses[b.species], b.atom_ptr, 600.0, 4242))
        m.md_init(s, nl, mp, st)
        m.md_run(s, nl, mp, st, args.repeat)
        m.check_status()
        torch.cuda.synchronize()
        print(f"ok md {args.workload} atoms={b.n_atoms} steps={args.repeat} builds={int(st.n_builds.item())}")
        return
    nl = m.build_neighbors(s)
    if args.op == "neighbors":
        for _ in range(args.repeat):
            m.build_neighbors(s, nl, check=False)
    elif args.op == "ef":
        for _ in range(args.repeat + 1):
            m.energy_forces(s, nl)
    else:
        E, F, _ = m.energy_forces(s, nl)
        gE = torch.ones_like(E)
        gF = torch.full_like(F, 0.01)
        for _ in range(args.repeat + 1):
            m.param_grad(s, nl, gE, gF)
    m.check_status()
    torch.cuda.synchronize()
    print(f"ok {args.op} {args.workload} atoms={b.n_atoms} pairs={int(nl.n_pairs.item())} precision={args.precision}")


if __name__ == "__main__":
    main()
