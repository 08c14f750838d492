"""Host logic of the solve-plan cache (no GPU): keys, storing, and the
choice between a cached plan and a fresh tuning."""
import json

from paper_1910_01260_gb300 import tuning


class StubModel:
    def __init__(self):
        self.installed = []
        self.tuned = 0

    def st_rom_solve_set_plan(self, precision, plan):
        self.installed.append((precision, plan))

    def st_rom_solve_tune(self, n_mu, theta, ns_nt, uhat, reps=2):
        self.tuned += 1
        return {"best": {"panel": 16, "ctas_per_sm": 3, "order": 0}, "best_ms": 20.0, "default_ms": 27.0,
                "n_candidates": 37, "candidates": [{"panel": 16, "ctas_per_sm": 3, "order": 0, "ms": 20.0}]}


def test_key_depends_on_the_size_classes_not_their_order():
    a = tuning.plan_key("GB300", 40, 12, 2, 3, 4096, [(10, 4), (40, 12), (10, 4)])
    b = tuning.plan_key("GB300", 40, 12, 2, 3, 4096, [(40, 12), (10, 4)])
    c = tuning.plan_key("GB300", 40, 12, 2, 3, 4096, [(40, 12)])
    assert a == b and a != c
    assert tuning.plan_key("GB300", 40, 12, 2, 3, 4096) != a


def test_load_or_tune_tunes_once_then_uses_the_cache(tmp_path):
    path = str(tmp_path / "plans.json")
    m = StubModel()
    e1 = tuning.load_or_tune(m, "k", 2, 8, None, None, None, path=path)
    assert e1["source"] == "tuned" and m.tuned == 1 and e1["plan"]["panel"] == 16
    stored = json.load(open(path))
    assert stored["k"]["plan"] == {"panel": 16, "ctas_per_sm": 3, "order": 0}
    assert stored["k"]["default_ms"] == 27.0 and "candidates" not in stored["k"]
    e2 = tuning.load_or_tune(m, "k", 2, 8, None, None, None, path=path)
    assert e2["source"] == "cache" and m.tuned == 1
    assert m.installed == [(2, {"panel": 16, "ctas_per_sm": 3, "order": 0})]


def test_a_damaged_cache_is_ignored(tmp_path):
    path = tmp_path / "plans.json"
    path.write_text("{not json")
    assert tuning.load(str(path)) == {}
    m = StubModel()
    assert tuning.load_or_tune(m, "k", 2, 8, None, None, None, path=str(path))["source"] == "tuned"
