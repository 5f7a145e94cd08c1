"""Shared helpers of the GPU parity tests (error metrics and batch slicing)."""
import numpy as np

from synth.systems import make_batch

# Tolerances stated for the path: FP32 within 1e-5 relative on energy/atom and force RMS;
# mixed (BF16 network) within 2e-3.
TOL = {"fp32": 1e-5, "mixed": 2e-3}
# Element-wise bound, as a multiple of the norm tolerance times the reference force RMS.
ELEMENT_FACTOR = 20.0


def subset(batch, idx):
    """Batch made of the structures ``idx`` of ``batch``."""
    ap = batch.atom_ptr
    structs = [(batch.pos[ap[b]:ap[b + 1]], batch.species[ap[b]:ap[b + 1]], batch.cell[b]) for b in idx]
    return make_batch(structs, batch.n_species)


def energy_error(E, ref, batch):
    """max over structures of |E_b - E_b^ref| / N_b, divided by the RMS atomic energy of b."""
    worst = 0.0
    ap = batch.atom_ptr
    for b in range(batch.n_structures):
        n = ap[b + 1] - ap[b]
        if n == 0:
            assert abs(E[b]) == 0.0
            continue
        scale = np.sqrt((ref["E_atom"][ap[b]:ap[b + 1]] ** 2).mean())
        worst = max(worst, abs(E[b] - ref["E"][b]) / n / scale)
    return worst


def force_error(F, ref):
    """RMS(F - F_ref) / RMS(F_ref) and the largest element-wise error in units of RMS(F_ref)."""
    rms = np.sqrt((ref["F"] ** 2).mean())
    d = F - ref["F"]
    return np.sqrt((d ** 2).mean()) / rms, np.abs(d).max() / rms


def virial_error(W, ref):
    return np.abs(W - ref["virial"]).max() / np.abs(ref["virial"]).max()
