"""Host logic of the launch-shape autotuner: coordinate descent over the knobs and the JSON
cache (a fake model with a synthetic cost stands in for the GPU timing)."""
import json

from paper_2505_22168_b300 import autotune


class FakeModel:
    precision = "mixed"

    def __init__(self):
        self.tuning = {}

    def set_tuning(self, **knobs):
        self.tuning.update({k: v for k, v in knobs.items() if v is not None})


def cost(m):
    t = m.tuning
    # separable cost with its minimum at nl_items=1, nl_split=4, pair_tpa=8, forces_tpa=16,
    # gemm_bn=128, gemm_cps=2
    return (1.0 + abs(t.get("nl_items", 0) - 1) + 0.1 * abs(t.get("nl_split", 0) - 4)
            + 0.01 * abs(t.get("pair_tpa", 0) - 8) + 0.005 * abs(t.get("forces_tpa", 0) - 16)
            + 0.001 * abs(t.get("gemm_bn", 0) - 128) + 0.0001 * abs(t.get("gemm_cps", 0) - 2))


def test_coordinate_descent_finds_the_separable_minimum():
    m = FakeModel()
    r = autotune.tune(m, None, None, None, timer=cost, key="k")
    assert r["settings"] == {"nl_items": 1, "nl_split": 4, "pair_tpa": 8, "forces_tpa": 16, "gemm_bn": 128,
                             "gemm_cps": 2, "mlp_cluster": 0}
    assert m.tuning == r["settings"]
    assert r["ms"] == min(ms for _, ms in r["trials"])
    assert r["default_ms"] == r["trials"][0][1]


def test_fp32_models_skip_the_tensor_core_knob():
    m = FakeModel()
    m.precision = "fp32"
    r = autotune.tune(m, None, None, None, timer=cost, key="k")
    assert "gemm_bn" not in r["settings"] and "gemm_cps" not in r["settings"] and "mlp_cluster" not in r["settings"]


def test_cache_round_trip(tmp_path):
    path = tmp_path / "tune.json"
    m = FakeModel()
    r1 = autotune.tune(m, None, None, None, timer=cost, key="sys-a", cache=path)
    assert not r1["cached"]
    table = json.loads(path.read_text())
    assert table["sys-a"]["settings"] == r1["settings"]
    calls = []
    m2 = FakeModel()
    r2 = autotune.tune(m2, None, None, None, timer=lambda mm: calls.append(1) or 0.0, key="sys-a", cache=path)
    assert r2["cached"] and not calls
    assert m2.tuning == r1["settings"]
