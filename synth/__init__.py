"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmarks.

This package only draws random numbers and lays out atoms; it contains none of the
model's arithmetic (no basis functions, moments, contractions or network).  Both the
FP64 oracle (``oracle/``) and the GPU library (``paper_2505_22168_b300``) consume what it
produces; neither is imported from here.
"""
from .systems import (  # noqa: F401
    Batch,
    emim_box,
    li3po4_crystal,
    li3po4_random,
    make_batch,
    dimer,
    EMIM_SPECIES,
    LI3PO4_SPECIES,
)
from .params import make_params, param_shapes  # noqa: F401
from .configs import config, CONFIGS  # noqa: F401
