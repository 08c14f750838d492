"""Pins of the oracle's full-order march (Eq. fom) and space-time form (Eq. st-fom)."""
import numpy as np
import pytest

from oracle import fom
from workloads import make_problem, problem_for


def _A(p, mu):
    return fom.affine_operator(p.rowptr, p.col, p.vals, p.theta(mu))


def test_solvers_agree_c1():
    p = problem_for("c1")
    A = _A(p, p.test_mu[0])
    dt, F = p.dt[:12], p.F[:12]
    U1 = fom.fom_march(A, dt, p.B, F, p.u0, solver="splu")
    U2 = fom.fom_march(A, dt, p.B, F, p.u0, solver="dense")
    U3 = fom.fom_march(A, dt, p.B, F, p.u0, solver="bicgstab", tol=1e-15)
    s = np.abs(U1).max()
    assert np.abs(U1 - U2).max() / s < 1e-13
    assert np.abs(U1 - U3).max() / s < 1e-12


def test_march_equals_spacetime_system():
    # Eq. st-fom is the same problem solved all at once.
    p = make_problem(dim=2, M=4, quad="s4", Nt=5, u0="seeded", g="sin")
    A = _A(p, np.array([0.9, 0.6]))
    U = fom.fom_march(A, p.dt, p.B, p.F, p.u0)
    Ust = fom.st_fom_solve(A, p.dt, p.B, p.F, p.u0)
    assert np.abs(U - Ust).max() / np.abs(U).max() < 1e-13
    Ast, rhs = fom.st_fom_system(A, p.dt, p.B, p.F, p.u0)
    # block structure: diagonal blocks I - dt A, sub-diagonal -I
    n = p.N
    blk = Ast[n:2 * n, 0:n].toarray()
    assert np.allclose(blk, -np.eye(n))
    assert np.allclose(Ast[0:n, 0:n].toarray(), np.eye(n) - p.dt[0] * A.toarray())


@pytest.mark.parametrize("mu1", [0.5, 1.3])
def test_pure_absorption_closed_form(mu1):
    # Streaming off, no scattering, homogeneous medium: A = -v sigma_t I and
    # backward Euler gives u^n = (1 + dt v sigma_t)^(-n) u0.
    p = make_problem(dim=1, M=16, quad="gl4", Nt=20, rho="homogeneous", source="none",
                     streaming=False, u0="seeded")
    A = _A(p, np.array([mu1, 0.0]))
    U = fom.fom_march(A, p.dt, p.B, p.F, p.u0)
    for n in (1, 7, 20):
        ref = (1.0 + p.dt[0] * mu1) ** (-n) * p.u0
        assert np.abs(U[:, n - 1] - ref).max() < 1e-14


def test_scattering_closed_form_isotropic():
    # With an isotropic state, P u = u (sum w = 1), so the loss rate is
    # sigma_t (1 - c): u^n = (1 + dt v sigma_t (1 - c))^(-n) u0.
    p = make_problem(dim=2, M=4, quad="s4", Nt=10, rho="homogeneous", source="none",
                     streaming=False, u0="isotropic")
    mu1, c = 1.2, 0.7
    A = _A(p, np.array([mu1, c]))
    U = fom.fom_march(A, p.dt, p.B, p.F, p.u0)
    ref = (1.0 + p.dt[0] * mu1 * (1 - c)) ** (-10) * p.u0
    assert np.abs(U[:, -1] - ref).max() < 1e-14


def test_source_recursion_closed_form():
    # Streaming off, isotropic source, zero start: every cell follows
    # u^n = (u^{n-1} + dt v q g(t_n)) / (1 + dt v sigma_t (1 - c)).
    p = make_problem(dim=1, M=64, quad="gl8", Nt=25, source="box", g="sin", streaming=False)
    mu = np.array([0.8, 0.3])
    A = _A(p, mu)
    U = fom.fom_march(A, p.dt, p.B, p.F, p.u0)
    sig_a = mu[0] * np.tile(p.rho, p.L) * (1 - mu[1])
    q = p.B[:, 0]
    u = np.zeros(p.N)
    for n in range(p.Nt):
        u = (u + p.dt[n] * q * p.F[n, 0]) / (1.0 + p.dt[n] * sig_a)
        assert np.abs(U[:, n] - u).max() < 1e-14 * max(1.0, np.abs(u).max())


def test_nonuniform_steps():
    # t_k = sum dt_j; the march takes dt_k per step (Eq. fom).
    p = make_problem(dim=1, M=8, quad="gl4", Nt=6, rho="homogeneous", source="none",
                     streaming=False, u0="seeded")
    dt = np.array([0.1, 0.3, 0.05, 0.2, 0.15, 0.2])
    A = _A(p, np.array([1.0, 0.0]))
    U = fom.fom_march(A, dt, p.B, p.F, p.u0)
    ref = p.u0 / np.prod(1.0 + dt)
    assert np.abs(U[:, -1] - ref).max() < 1e-15


def test_bicgstab_polynomial_initial_iterate():
    # With A = 0 the march is u^k = u^{k-1} + dt B f^k; choosing f so that u^k
    # is a cubic in k, the extrapolation of degree >= 3 through the previous
    # levels is exact, so BiCGSTAB starts converged (0 iterations) from the
    # fifth step on, while from the previous level it needs one iteration.
    n, nt = 6, 10
    rng = np.random.default_rng(2)
    c = rng.standard_normal((4, n))
    ks = np.arange(nt + 1, dtype=float)
    traj = np.stack([c[0] + c[1] * k + c[2] * k ** 2 + c[3] * k ** 3 for k in ks])  # u^0..u^nt
    dt = np.ones(nt)
    B = np.eye(n)
    F = traj[1:] - traj[:-1]
    A = fom.sp.csr_matrix((n, n))
    for order, want in ((4, 0), (0, 1)):
        its = []
        U = fom.fom_march(A, dt, B, F, traj[0], solver="bicgstab", tol=1e-12, iters=its, x0_order=order)
        assert np.abs(U.T - traj[1:]).max() < 1e-9 * np.abs(traj).max()
        assert all(i == want for i in its[4:]), its
    # and on a transport problem the solution does not depend on it
    p = problem_for("c1")
    A = _A(p, p.test_mu[0])
    U1 = fom.fom_march(A, p.dt[:12], p.B, p.F[:12], p.u0, solver="splu")
    its0, its4 = [], []
    U0 = fom.fom_march(A, p.dt[:12], p.B, p.F[:12], p.u0, solver="bicgstab", tol=1e-14, iters=its0)
    U4 = fom.fom_march(A, p.dt[:12], p.B, p.F[:12], p.u0, solver="bicgstab", tol=1e-14, iters=its4, x0_order=4)
    s = np.abs(U1).max()
    assert np.abs(U0 - U1).max() / s < 1e-12 and np.abs(U4 - U1).max() / s < 1e-12
    assert sum(its4) < sum(its0)
