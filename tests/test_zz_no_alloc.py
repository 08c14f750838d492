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


def _model():
    p = make_problem(dim=2, M=8, quad="s4", Nt=20, source="gaussian", g="ramp", ns=12, nt=5)
    rng = np.random.default_rng(9)
    Phi = np.linalg.qr(rng.standard_normal((p.N, p.ns)))[0]
    T = np.zeros((p.Nt, p.ns * p.nt))
    for i in range(p.ns):
        T[:, i::p.ns] = np.linalg.qr(rng.standard_normal((p.Nt, p.nt)))[0]
    m = make_model(p)
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
