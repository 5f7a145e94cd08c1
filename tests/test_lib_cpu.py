"""CPU checks of the C-ABI library: it loads, exports every symbol include/gm.h declares,
and its host-side logic (parameter count, argument validation, status strings) works
without a GPU.  No compute call is made."""
import re
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def lib():
    from paper_2505_22168_b300 import build
    build.build()
    from paper_2505_22168_b300 import _lib
    return _lib


def _declared():
    text = (ROOT / "include" / "gm.h").read_text()
    return sorted(set(re.findall(r"^GM_API\s+[^;]*?\b(gm_\w+)\s*\(", text, flags=re.M)))


def test_exports_every_declared_symbol(lib):
    import subprocess
    declared = _declared()
    assert len(declared) >= 13
    out = subprocess.run(["nm", "-D", "--defined-only", str(lib.LIB_PATH)], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (gm_\w+)", out))
    assert set(declared) <= exported, set(declared) - exported
    assert exported == set(declared), exported - set(declared)
    assert set(lib.EXPORTS) == set(declared)
    L = lib.load()
    for name in declared:
        getattr(L, name)


def test_param_count_matches_layout(lib):
    import synth
    for S, H in ((5, 128), (3, 512), (1, 64)):
        d = lib.GmModelDesc(S, 7, 5, H, 1, 0, 0.5, 5.0)
        n = sum(int(np.prod(s)) for s in synth.param_shapes(S, H).values())
        assert lib.gm_param_count(d) == n == 35 * S * S + 360 * H + H + H * H + H + H + 1 + 2 * S


@pytest.mark.parametrize("bad,code", [
    (dict(n_radial=4), 3), (dict(n_basis=8), 3), (dict(n_hidden=96), 3), (dict(n_hidden=1024), 3),
    (dict(n_species=17), 3), (dict(activation=5), 1), (dict(precision=7), 1), (dict(r_cut=0.3), 1),
])
def test_model_create_rejects_unsupported(lib, bad, code):
    f = dict(n_species=5, n_basis=7, n_radial=5, n_hidden=128, activation=1, precision=0, r_min=0.5, r_cut=5.0)
    f.update(bad)
    d = lib.GmModelDesc(*f.values())
    with pytest.raises(lib.GmError) as e:
        lib.gm_model_create(d)
    assert e.value.code == code


def test_status_strings(lib):
    assert lib.gm_status_string(0) == "ok"
    assert "capacity" in lib.gm_status_string(2)
    assert lib.gm_status_string(99) == "unknown status"


def test_null_arguments_rejected_on_host(lib):
    L = lib.load()
    assert L.gm_build_neighbors(None, None, None, None, 0, None, None) == lib.GM_ERR_ARG
    assert L.gm_energy_forces(None, None, None, None, None, None, None, 0, None, None) == lib.GM_ERR_ARG
    assert L.gm_status_clear(None, None) == lib.GM_ERR_ARG


def test_header_constants_match_binding(lib):
    text = (ROOT / "include" / "gm.h").read_text()
    assert int(re.search(r"#define GM_MAX_ATOMS (\d+)", text).group(1)) == lib.GM_MAX_ATOMS
    tune = dict(re.findall(r"(GM_TUNE_\w+) = (\d+)", text))
    assert tune and all(int(v) == getattr(lib, k) for k, v in tune.items())
