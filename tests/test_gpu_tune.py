"""The batched solve's launch plans and their autotuner on the GPU: every
plan solves the batch to the same results (bit for bit at equal panel width),
the tuner installs the fastest candidate, and invalid plans are refused."""
import numpy as np
import pytest

from gpu_util import dev_B, dev_tensor, make_model, rel_max
from workloads import make_problem

pytestmark = pytest.mark.gpu


def _model(precision, refine):
    p = make_problem(dim=2, M=8, quad="s4", Nt=20, source="gaussian", g="ramp", ns=40, nt=12)
    rng = np.random.default_rng(5)
    Phi = np.linalg.qr(rng.standard_normal((p.N, p.ns)))[0]
    T = np.zeros((p.Nt, p.ns * p.nt))
    for i in range(p.ns):
        T[:, i::p.ns] = np.linalg.qr(rng.standard_normal((p.Nt, p.nt)))[0]
    m = make_model(p, precision=precision, refine_steps=refine)
    m.st_model_set_basis(p.ns, p.nt, p.Nt, dev_tensor(Phi.T.copy()), dev_tensor(T.T.copy()))
    m.st_rom_assemble(p.dt, dev_B(p), p.F, None)
    return p, m


def _batch(p, n, seed=3):
    rng = np.random.default_rng(seed)
    mu = p.mu_lo + rng.random((n, 2)) * (p.mu_hi - p.mu_lo)
    choices = np.array([(10, 4), (20, 8), (30, 10), (40, 12)], dtype=np.int32)
    return dev_tensor(p.theta(mu)), dev_tensor(choices[rng.integers(0, 4, n)])


@pytest.mark.parametrize("precision,refine", [(0, 1), (2, 3)])
def test_plans_give_the_same_solutions(precision, refine):
    torch = __import__("torch")
    p, m = _model(precision, refine)
    th, sz = _batch(p, 300)
    nf = p.ns * p.nt
    out = {}
    for plan in (None, {"panel": 16, "ctas_per_sm": 1, "order": 0}, {"panel": 16, "ctas_per_sm": 2, "order": 1},
                 {"panel": 16, "ctas_per_sm": 1, "order": 2}, {"panel": 8, "ctas_per_sm": 2, "order": 2}):
        m.st_rom_solve_set_plan(precision, plan)
        uh = torch.zeros((300, nf), dtype=torch.float64, device="cuda:0")
        st_ = torch.full((300,), -1, dtype=torch.int32, device="cuda:0")
        m.st_rom_solve(300, th, sz, uh, None, st_)
        m.st_sync()
        assert int((st_ != 0).sum()) == 0
        out[str(plan)] = uh.cpu().numpy()
        if plan is not None:
            got = m.st_rom_solve_get_plan(precision)
            assert got["panel"] == plan["panel"] and got["order"] == plan["order"]
            assert 1 <= got["ctas_per_sm"] <= plan["ctas_per_sm"]
    ref = out["None"]
    same_panel = [k for k in out if "'panel': 16" in k]
    for k in same_panel[1:]:
        assert np.array_equal(out[k], out[same_panel[0]])      # panel fixed: bit for bit
    for k, v in out.items():
        assert rel_max(v, ref) < 1e-10
    m.close()


def test_tuner_installs_the_fastest_candidate():
    torch = __import__("torch")
    import paper_1910_01260_gb300 as st
    p, m = _model(st.ST_FP32_LU, 3)
    th, sz = _batch(p, 400)
    uh = torch.zeros((400, p.ns * p.nt), dtype=torch.float64, device="cuda:0")
    r = m.st_rom_solve_tune(400, th, sz, uh, reps=1)
    assert r["n_candidates"] >= 4 and len(r["candidates"]) == r["n_candidates"]
    assert r["best_ms"] == min(c["ms"] for c in r["candidates"])
    assert r["default_ms"] == r["candidates"][0]["ms"] >= r["best_ms"]
    got = m.st_rom_solve_get_plan(st.ST_FP32_LU)
    if r["best"]["panel"]:
        assert got["panel"] == r["best"]["panel"] and got["order"] == r["best"]["order"]
    # the FP64 plan is untouched
    assert m.st_rom_solve_get_plan(st.ST_FP64)["order"] == st.ST_ORDER_LARGEST_FIRST
    with pytest.raises(st.StError) as e:
        m.st_rom_solve_set_plan(st.ST_FP32_LU, {"panel": 12, "ctas_per_sm": 1, "order": 0})
    assert e.value.code == st.ST_ERR_ARG
    with pytest.raises(st.StError):
        m.st_rom_solve_set_plan(st.ST_FP32_LU, {"panel": 16, "ctas_per_sm": 1, "order": 7})
    m.close()
