"""GPU parity of the full-order snapshot march (Eq. fom) against the oracle.

Tolerance: both sides solve every step to a relative residual of 1e-13
(GPU BiCGSTAB) or exactly (oracle sparse LU); with cond(I - dt A) = O(10)
the per-step error is ~1e-12 and the march stays below 1e-10 relative to
max |u| (the FP64 bar of the method)."""
import numpy as np
import pytest

from gpu_util import gpu_fom, make_model, oracle_fom, rel_max
from oracle import fom
from workloads import make_problem, problem_for

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(params=[1, 2], ids=["grid", "cluster"])
def path(request):
    """st_options.fom_path: the cooperative grid march (ST_FOM_GRID) and the
    cluster-per-sample march (ST_FOM_CLUSTER)."""
    return request.param


def test_fom_c1_all_samples(path):
    p = problem_for("c1")
    mus = np.concatenate([p.train_mu, p.test_mu])       # 12 samples: padded group of 16
    m = make_model(p, fom_path=path)
    got, status, _ = gpu_fom(m, p, mus)
    assert (status == 0).all()
    ref = oracle_fom(p, mus)
    for g, r in zip(got, ref):
        assert rel_max(g, r) < TOL
    m.close()


@pytest.mark.parametrize("n_mu", [1, 2, 3, 33])
def test_fom_group_shapes(n_mu, path):
    # one sample (scalar path), padding inside a group, and two groups
    p = make_problem(dim=2, M=8, quad="s4", Nt=7, source="gaussian", g="ramp", u0="seeded")
    mus = p.mu_lo + np.random.default_rng(n_mu).random((n_mu, 2)) * (p.mu_hi - p.mu_lo)
    m = make_model(p, fom_path=path)
    got, status, _ = gpu_fom(m, p, mus, u0=p.u0)
    assert (status == 0).all()
    ref = oracle_fom(p, mus, u0=p.u0)
    for g, r in zip(got, ref):
        assert rel_max(g, r) < TOL
    m.close()


def test_fom_c2_first_steps(path):
    p = problem_for("c2")
    mus = p.train_mu
    m = make_model(p, fom_path=path)
    got, status, it = gpu_fom(m, p, mus, Nt=12, with_iters=True)
    assert (status == 0).all()
    ref = oracle_fom(p, mus[:3], Nt=12)
    for g, r in zip(got[:3], ref):
        assert rel_max(g, r) < TOL
    # iteration counts are those of textbook BiCGSTAB on the same systems,
    # started from the same quartic extrapolation of the previous levels
    A = fom.affine_operator(p.rowptr, p.col, p.vals, p.theta(mus[0]))
    its = []
    fom.fom_march(A, p.dt[:12], p.B, p.F[:12], None, solver="bicgstab", tol=1e-13, iters=its, x0_order=4)
    assert np.abs(it[:, 0] - np.array(its)).max() <= 1
    m.close()


def test_fom_pure_absorption_closed_form(path):
    p = make_problem(dim=1, M=16, quad="gl4", Nt=20, rho="homogeneous", source="none",
                     streaming=False, u0="seeded")
    mus = np.array([[0.5, 0.0], [1.3, 0.0]])
    m = make_model(p, fom_path=path)
    got, status, _ = gpu_fom(m, p, mus, u0=p.u0)
    assert (status == 0).all()
    for g, mu in zip(got, mus):
        for n in (1, 9, 20):
            ref = (1.0 + p.dt[0] * mu[0]) ** (-n) * p.u0
            assert np.abs(g[:, n - 1] - ref).max() < 1e-13
    m.close()


def test_fom_zero_input_gives_zero_state(path):
    p = make_problem(dim=2, M=8, quad="s4", Nt=5, source="none")
    m = make_model(p, fom_path=path)
    got, status, _ = gpu_fom(m, p, p.train_mu)
    assert (status == 0).all()
    assert all(np.abs(g).max() == 0.0 for g in got)
    m.close()


def test_fom_iteration_limit_reported(path):
    import paper_1910_01260_gb300 as st
    p = make_problem(dim=2, M=8, quad="s4", Nt=4, source="gaussian")
    m = make_model(p, maxit=1, fom_path=path)
    got, status, _ = gpu_fom(m, p, p.train_mu)
    assert (status == st.ST_ERR_NOT_CONVERGED).all()
    with pytest.raises(st.StError) as e:
        m.st_sync()
    assert e.value.code == st.ST_ERR_NOT_CONVERGED
    m.st_sync()   # cleared
    m.close()


def test_fom_nonfinite_sample_isolated(path):
    import paper_1910_01260_gb300 as st
    p = make_problem(dim=2, M=8, quad="s4", Nt=4, source="gaussian")
    torch = __import__("torch")
    m = make_model(p, fom_path=path)
    theta = p.theta(p.train_mu)
    theta[1, 1] = np.nan
    snaps = torch.zeros((4, p.Nt, p.N), dtype=torch.float64, device="cuda:0")
    status = torch.full((4,), -1, dtype=torch.int32, device="cuda:0")
    from gpu_util import dev_B
    m.st_fom_march(theta, p.dt, None, dev_B(p), p.F, snaps, None, status)
    torch.cuda.synchronize()
    s = status.cpu().numpy()
    assert s[1] == st.ST_ERR_NONFINITE and s[0] == s[2] == s[3] == 0
    ref = oracle_fom(p, p.train_mu[[0, 2]])
    S = snaps.cpu().numpy()
    assert rel_max(S[0].T, ref[0]) < TOL and rel_max(S[2].T, ref[1]) < TOL
    with pytest.raises(st.StError):
        m.st_sync()
    m.close()


def test_fom_deterministic(path):
    p = make_problem(dim=2, M=16, quad="s4", Nt=6, source="gaussian")
    m = make_model(p, fom_path=path)
    a, _, _ = gpu_fom(m, p, p.train_mu)
    b, _, _ = gpu_fom(m, p, p.train_mu)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    m.close()


def test_fom_term_split_random_affine_operator(path):
    """A random 3-term affine operator whose entries have one, two or three
    nonzero terms (and some explicit all-zero entries): the march's
    term-split operator (shared single-term values scaled by theta_q, per
    sample values where terms overlap) against the oracle's CSR."""
    import types
    rng = np.random.default_rng(11)
    N, Q, Nt = 300, 3, 8
    rows, cols = [], []
    for r in range(N):
        nb = rng.choice(N, size=7, replace=False)
        cs = np.unique(np.concatenate([[r], nb]))
        rows += [r] * len(cs)
        cols += list(cs)
    rows, cols = np.array(rows), np.array(cols)
    nnz = len(rows)
    mask = rng.random((Q, nnz)) < 0.5
    mask[:, rows == cols] = True                       # diagonal in every term
    mask[:, rng.random(nnz) < 0.05] = False            # explicit all-zero entries
    vals = rng.standard_normal((Q, nnz)) * mask * 0.3
    diag = rows == cols
    vals[:, diag] = -np.abs(vals[:, diag]) - 2.0       # dissipative diagonal
    rowptr = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=N))]).astype(np.int64)
    Bm = rng.standard_normal((N, 1))
    dt = np.full(Nt, 0.05)
    F = np.sin(np.arange(1, Nt + 1) * 0.3)[:, None]
    p = types.SimpleNamespace(N=N, rowptr=rowptr, col=cols.astype(np.int32), vals=vals, B=Bm, F=F, dt=dt,
                              Nt=Nt, theta=lambda t: np.asarray(t, dtype=np.float64))
    thetas = np.array([[1.0, 0.7, 0.3], [1.0, 1.3, 0.9], [0.5, 0.2, 1.1]])
    m = make_model(p, fom_path=path)
    got, status, _ = gpu_fom(m, p, thetas)
    assert (status == 0).all()
    for k, th in enumerate(thetas):
        A = fom.affine_operator(p.rowptr, p.col, p.vals, th)
        ref = fom.fom_march(A, dt, Bm, F, None)
        assert rel_max(got[k], ref) < TOL
    m.close()


def test_fom_barrier_wait_runs_out_and_model_recovers():
    # A grid barrier allowed a single poll gives up (no CTA can arrive in
    # time): the march stops with ST_ERR_TIMEOUT instead of hanging, and the
    # same model marches normally once the limit is restored.  The march has
    # no asynchronous copies in flight, so CTAs that stop early leave nothing
    # behind.
    import paper_1910_01260_gb300 as st
    p = make_problem(dim=2, M=8, quad="s4", Nt=4, source="gaussian", g="ramp")
    mus = p.train_mu[:3]
    m = make_model(p, spin_limit=1, fom_path=1)   # grid barriers
    with pytest.raises(st.StError) as e:
        gpu_fom(m, p, mus)
        m.st_sync()
    assert e.value.code == st.ST_ERR_TIMEOUT
    m.st_sync()  # the error word was read and cleared
    m.st_model_set_options(spin_limit=20000000)
    got, status, _ = gpu_fom(m, p, mus)
    assert (status == 0).all()
    ref = oracle_fom(p, mus, Nt=4)
    for g, r in zip(got, ref):
        assert rel_max(g, r) < TOL
    m.close()


def test_fom_cluster_matches_grid_at_full_size():
    """The two march kernels on the 2-D S4 operator of N = 49,152 (16
    training parameters, 30 steps): same iteration counts within one and the
    same snapshots to the march tolerance; the cluster march's first steps
    against the oracle's sparse LU."""
    p = problem_for("c4")
    Nt = 30
    out = {}
    for path in (1, 2):
        m = make_model(p, fom_path=path)
        got, status, it = gpu_fom(m, p, p.train_mu, Nt=Nt, with_iters=True)
        assert (status == 0).all()
        out[path] = (got, it)
        m.close()
    for a, b in zip(out[1][0], out[2][0]):
        assert rel_max(b, a) < TOL
    assert np.abs(out[1][1] - out[2][1]).max() <= 1
    ref = oracle_fom(p, p.train_mu[:2], Nt=Nt)
    for g, r in zip(out[2][0][:2], ref):
        assert rel_max(g, r) < TOL


def test_fom_cluster_path_rejects_an_operator_too_large_for_it():
    import paper_1910_01260_gb300 as st
    # N = 72 x 72 cells x 12 directions = 62,208: one CTA's share of four vectors is 243 KB
    p = make_problem(dim=2, M=72, quad="s4", Nt=2, source="gaussian")   # N = 62,208
    m = make_model(p, fom_path=2)
    with pytest.raises(st.StError) as e:
        gpu_fom(m, p, p.train_mu[:1])
    assert e.value.code == st.ST_ERR_ARG
    m.close()
