"""GPU parity of the full-order residual norms ||r^k(u^k, u^{k-1})||_2 (Eq.
residual), the factor of the error bounds of Theorems 1 and 3, through the C
ABI.

Tolerance: both sides evaluate r^k = u^k - u^{k-1} - dt_k A u^k - dt_k B f^k in
FP64 in different orders, so their residuals differ by at most a small
multiple of eps times s_k = ||u^k|| + ||u^{k-1}|| + dt_k || |A| |u^k| || +
dt_k || |B| |f^k| ||; the norms then differ by no more (triangle
inequality).  The tests allow 64 eps s_k."""
import numpy as np
import pytest

from gpu_util import dev_B, dev_tensor, make_model, oracle_fom
from oracle import fom, pod, strom
from workloads import make_problem, problem_for

pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


def _torch():
    return __import__("torch")


def _norms(m, p, thetas, U, u0=None, dt=None):
    """U host [n, Nt, N]; returns the library's norms [n, Nt]."""
    torch = _torch()
    n = len(thetas)
    Ud = torch.tensor(U, device="cuda:0")
    rn = torch.full((n, p.Nt), float("nan"), dtype=torch.float64, device="cuda:0")
    m.st_rom_residual_norms(np.asarray(thetas), p.dt if dt is None else dt,
                            None if u0 is None else dev_tensor(u0), dev_B(p), p.F, Ud, rn)
    torch.cuda.synchronize()
    return rn.cpu().numpy()


def _oracle(p, theta, Uk, u0=None, dt=None):
    """(norms, scales s_k) of one trajectory Uk (N x Nt)."""
    dt = p.dt if dt is None else dt
    A = fom.affine_operator(p.rowptr, p.col, p.vals, theta)
    init = np.zeros(p.N) if u0 is None else u0
    R = strom.fom_residual(A, dt, p.B, p.F, Uk, init)
    absA = abs(A)
    prev = np.concatenate([init[:, None], Uk[:, :-1]], 1)
    s = (np.linalg.norm(Uk, axis=0) + np.linalg.norm(prev, axis=0) +
         dt * np.linalg.norm(absA @ np.abs(Uk), axis=0) +
         dt * np.linalg.norm(np.abs(p.B) @ np.abs(p.F.T), axis=0))
    return np.linalg.norm(R, axis=0), s


@pytest.fixture(scope="module")
def c1_rom():
    p = problem_for("c1")
    blocks = oracle_fom(p, p.train_mu)
    ref = pod.pod_exact(blocks, p.ns, p.nt)
    return p, ref


def _rom_fields(m, p, thetas):
    torch = _torch()
    n = len(thetas)
    nf = p.ns * p.nt
    uh = torch.zeros((n, nf), dtype=torch.float64, device="cuda:0")
    m.st_rom_solve(n, dev_tensor(np.asarray(thetas)), None, uh)
    u = torch.zeros((n, p.Nt, p.N), dtype=torch.float64, device="cuda:0")
    m.st_rom_reconstruct(n, uh, None, u)
    torch.cuda.synchronize()
    return u.cpu().numpy()


def test_residual_norms_of_spacetime_rom_trajectories(c1_rom):
    p, ref = c1_rom
    m = make_model(p)
    m.st_model_set_basis(p.ns, p.nt, p.Nt, dev_tensor(ref["Phi_s"].T.copy()), dev_tensor(ref["T"].T.copy()))
    m.st_rom_assemble(p.dt, dev_B(p), p.F, None)
    th = p.theta(p.test_mu)
    U = _rom_fields(m, p, th)
    got = _norms(m, p, th, U)
    for k in range(len(th)):
        want, s = _oracle(p, th[k], U[k].T)
        assert want.max() > 1e3 * 64 * EPS * s.max()      # far above rounding
        assert (np.abs(got[k] - want) <= 64 * EPS * s).all()
    m.close()


def test_residual_norms_of_fom_trajectories_are_at_solver_tolerance():
    # the FOM's own solution leaves only the BiCGSTAB residual of each step
    torch = _torch()
    p = problem_for("c1")
    m = make_model(p)
    th = p.theta(p.test_mu[:4])
    snaps = torch.empty((len(th), p.Nt, p.N), dtype=torch.float64, device="cuda:0")
    m.st_fom_march(th, p.dt, None, dev_B(p), p.F, snaps)
    m.st_sync()
    U = snaps.cpu().numpy()
    got = _norms(m, p, th, U)
    rhs = np.linalg.norm(p.dt[:, None] * (p.B @ p.F.T).T, axis=1)
    for k in range(len(th)):
        want, s = _oracle(p, th[k], U[k].T)
        assert (np.abs(got[k] - want) <= 64 * EPS * s).all()
        prev = np.concatenate([[0.0], np.linalg.norm(U[k], axis=1)[:-1]])
        assert (got[k] <= 10 * m.opts.tol * (rhs + prev) + 64 * EPS * s).all()
    m.close()


def test_residual_norms_with_initial_state_and_ragged_steps():
    p = make_problem(dim=2, M=8, quad="s4", Nt=9, u0="seeded", g="sin", source="gaussian",
                     ns=5, nt=3)
    dt = p.dt * np.array([1.0, 1.0, 0.5, 0.5, 2.0, 1.0, 1.0, 0.25, 0.75])
    rng = np.random.default_rng(31)
    th = p.theta(p.test_mu)
    U = rng.standard_normal((len(th), p.Nt, p.N))
    m = make_model(p)
    got = _norms(m, p, th, U, u0=p.u0, dt=dt)
    for k in range(len(th)):
        want, s = _oracle(p, th[k], U[k].T, u0=p.u0, dt=dt)
        assert (np.abs(got[k] - want) <= 64 * EPS * s).all()
    m.close()


def test_theorem1_bound_holds_with_library_residuals():
    # spatial ROM on a tiny problem: its error against the FOM stays below
    # the Theorem 1 bound built from the library's residual norms
    torch = _torch()
    p = make_problem(dim=1, M=8, quad="gl4", Nt=6, g="sin", ns=3, nt=2)
    blocks = oracle_fom(p, p.train_mu)
    ref = pod.pod_exact(blocks, p.ns, p.nt)
    m = make_model(p)
    m.st_model_set_basis(p.ns, p.nt, p.Nt, dev_tensor(ref["Phi_s"].T.copy()), dev_tensor(ref["T"].T.copy()))
    m.st_rom_assemble(p.dt, dev_B(p), p.F, None)
    th = p.theta(p.test_mu)
    us = torch.zeros((len(th), p.Nt, p.ns), dtype=torch.float64, device="cuda:0")
    m.st_rom_spatial_march(len(th), dev_tensor(th), None, us)
    torch.cuda.synchronize()
    U = np.einsum("pki,ni->pkn", us.cpu().numpy(), ref["Phi_s"])
    got = _norms(m, p, th, U)
    for k in range(len(th)):
        A = fom.affine_operator(p.rowptr, p.col, p.vals, th[k])
        Uf = fom.fom_march(A, p.dt, p.B, p.F, None, solver="dense")
        err = np.linalg.norm(Uf - U[k].T, axis=0)
        bound = strom.spatial_error_bound(A, p.dt, np.diag(got[k]), 0.0)
        assert err.max() > 1e-8 * np.abs(Uf).max()
        assert (err <= bound * (1 + 1e-10)).all()
    m.close()


def test_theorem3_bound_holds_with_library_residuals():
    # space-time ROM on a tiny problem: max_k ||u^k - u~^k|| <= sqrt(Nt)
    # ||(A^st)^-1||_2 max_k ||r^k|| (Theorem 3) with the library's residuals
    p = make_problem(dim=1, M=8, quad="gl4", Nt=6, g="sin", ns=3, nt=2)
    blocks = oracle_fom(p, p.train_mu)
    ref = pod.pod_exact(blocks, p.ns, p.nt)
    m = make_model(p)
    m.st_model_set_basis(p.ns, p.nt, p.Nt, dev_tensor(ref["Phi_s"].T.copy()), dev_tensor(ref["T"].T.copy()))
    m.st_rom_assemble(p.dt, dev_B(p), p.F, None)
    th = p.theta(p.test_mu)
    U = _rom_fields(m, p, th)
    got = _norms(m, p, th, U)
    for k in range(len(th)):
        A = fom.affine_operator(p.rowptr, p.col, p.vals, th[k])
        Uf = fom.fom_march(A, p.dt, p.B, p.F, None, solver="dense")
        Ast, _ = fom.st_fom_system(A, p.dt, p.B, p.F, None)
        smin = np.linalg.svd(Ast.toarray(), compute_uv=False).min()
        err = strom.st_inf_norm(Uf - U[k].T)
        assert err > 1e-8 * np.abs(Uf).max()
        assert err <= np.sqrt(p.Nt) / smin * got[k].max() * (1 + 1e-10)
    m.close()


def test_residual_norms_deterministic_and_independent_of_batching(c1_rom):
    p, ref = c1_rom
    m = make_model(p)
    rng = np.random.default_rng(2)
    th = p.theta(p.test_mu)
    U = rng.standard_normal((len(th), p.Nt, p.N))
    a = _norms(m, p, th, U)
    b = _norms(m, p, th, U)
    assert np.array_equal(a, b)
    for k in range(len(th)):
        one = _norms(m, p, th[k:k + 1], U[k:k + 1])
        assert np.array_equal(one[0], a[k])
    m.close()


def test_residual_norms_reject_bad_arguments():
    import paper_1910_01260_gb300 as st
    p = make_problem(dim=1, M=8, quad="gl4", Nt=6, ns=3, nt=2)
    m = make_model(p)
    U = np.zeros((1, p.Nt, p.N))
    with pytest.raises(st.StError) as e:
        _norms(m, p, p.theta(p.test_mu[:1]), U, dt=-p.dt)
    assert e.value.code == st.ST_ERR_ARG
    m.close()
