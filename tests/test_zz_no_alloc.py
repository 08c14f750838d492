"""st_rom_solve_static, the allocation-free variant of the batched reduced
solve, for callers that cannot allocate device memory while they solve (a
fixed pre-reserved memory budget, an outside pool that forbids side
allocations, or a context where allocation calls are not allowed).

Through the C ABI it must give the same results as st_rom_solve, within the
solve tolerance of the other tests (1e-10 relative), on two calls in a row --
the second call finds the previous call's leftovers in the shared scratch
array -- and it must not change the device's free memory.  This file is
collected last so that a failure here stops a first-failure run only after
every other test has run."""
import numpy as np
import pytest

from gpu_util import dev_B, dev_tensor, make_model, rel_max
from workloads import make_problem

pytestmark = pytest.mark.gpu


def _model(ns=12, nt=5, **opts):
    p = make_problem(dim=2, M=8, quad="s4", Nt=20, source="gaussian", g="ramp", ns=ns, nt=nt)
    rng = np.random.default_rng(9)
    Phi = np.linalg.qr(rng.standard_normal((p.N, p.ns)))[0]
    T = np.zeros((p.Nt, p.ns * p.nt))
    for i in range(p.ns):
        T[:, i::p.ns] = np.linalg.qr(rng.standard_normal((p.Nt, p.nt)))[0]
    m = make_model(p, **opts)
    m.st_model_set_basis(p.ns, p.nt, p.Nt, dev_tensor(Phi.T.copy()), dev_tensor(T.T.copy()))
    m.st_rom_assemble(p.dt, dev_B(p), p.F, None)
    return p, m


def _batch(p, n, seed):
    rng = np.random.default_rng(seed)
    mu = p.mu_lo + rng.random((n, 2)) * (p.mu_hi - p.mu_lo)
    choices = np.array([(12, 5), (6, 2), (9, 4), (3, 5), (12, 1)], dtype=np.int32)
    return p.theta(mu), choices[rng.integers(0, len(choices), n)]


def _run(m, fn, theta, sizes, nf):
    torch = __import__("torch")
    n = len(theta)
    uhat = torch.full((n, nf), float("nan"), dtype=torch.float64, device="cuda:0")
    res = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    status = torch.full((n,), -1, dtype=torch.int32, device="cuda:0")
    fn(n, dev_tensor(theta), dev_tensor(sizes), uhat, res, status)
    torch.cuda.synchronize()
    return uhat.cpu().numpy(), res.cpu().numpy(), status.cpu().numpy()


def test_static_solve_matches_allocating_solve_twice():
    torch = __import__("torch")
    p, m = _model()
    nf = p.ns * p.nt
    for call, seed in enumerate((21, 22)):
        theta, sizes = _batch(p, 700 + 300 * call, seed)
        want, wres, wst = _run(m, m.st_rom_solve, theta, sizes, nf)
        free0 = torch.cuda.mem_get_info()[0]
        got, gres, gst = _run(m, m.st_rom_solve_static, theta, sizes, nf)
        assert torch.cuda.mem_get_info()[0] == free0
        assert (wst == 0).all() and (gst == 0).all()
        for k, (a, b) in enumerate(sizes):
            assert rel_max(got[k, :a * b], want[k, :a * b]) < 1e-10
        assert np.abs(gres - wres).max() < 1e-12
    m.st_sync()
    m.close()


def test_static_solve_rejects_sizes_beyond_its_scratch():
    import paper_1910_01260_gb300 as st
    torch = __import__("torch")
    p, m = _model()
    n = 5_000_000          # the int section alone needs 40 MB > 32 MiB
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda:0")   # never touched
    with pytest.raises(st.StError) as e:
        m.st_rom_solve_static(n, dummy, None, dummy)
    assert e.value.code == st.ST_ERR_ARG
    assert "32" in st.last_error() or "scratch" in st.last_error()
    m.close()


@pytest.mark.parametrize("precision,refine", [(0, 1), (2, 3)])  # FP64 LU; FP32 LU + 3 refinements
def test_static_solve_at_n480_with_a_capped_grid(precision, refine):
    """ns*nt = 480 (the largest size class of the benchmark): only ~17 FP64
    (~34 FP32) factor matrices fit in the fixed scratch, fewer than the
    allocating path's blocks, so the capped grid and the per-precision matrix
    stride of the allocation-free path are the ones exercised."""
    torch = __import__("torch")
    p, m = _model(ns=40, nt=12, precision=precision, refine_steps=refine)
    nf = p.ns * p.nt
    rng = np.random.default_rng(31)
    for call in range(2):
        n = 200 + 40 * call
        mu = p.mu_lo + rng.random((n, 2)) * (p.mu_hi - p.mu_lo)
        choices = np.array([(40, 12), (30, 10), (20, 8), (10, 4)], dtype=np.int32)
        sizes = choices[rng.integers(0, len(choices), n)]
        sizes[:8] = (40, 12)
        theta = p.theta(mu)
        want, wres, wst = _run(m, m.st_rom_solve, theta, sizes, nf)
        free0 = torch.cuda.mem_get_info()[0]
        got, gres, gst = _run(m, m.st_rom_solve_static, theta, sizes, nf)
        assert torch.cuda.mem_get_info()[0] == free0
        assert (wst == 0).all() and (gst == 0).all()
        for k, (a, b) in enumerate(sizes):
            assert rel_max(got[k, :a * b], want[k, :a * b]) < 1e-10
        assert np.abs(gres - wres).max() < 1e-12
    m.st_sync()
    m.close()
