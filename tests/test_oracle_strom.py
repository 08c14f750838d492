"""Pins of the oracle's reduced models: space-time (Secs. 3.2, 4.3, 5.2) and
spatial (Secs. 3.1, 5.1)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import fom, pod, strom
from workloads import make_problem


@pytest.fixture(scope="module")
def tiny():
    p = make_problem(dim=1, M=8, quad="gl4", Nt=6, u0="seeded", g="sin", train=(2, 2),
                     ns=4, nt=3)
    blocks = [fom.fom_march(fom.affine_operator(p.rowptr, p.col, p.vals, p.theta(mu)),
                            p.dt, p.B, p.F, p.u0) for mu in p.train_mu]
    r = pod.pod_exact(blocks, p.ns, p.nt)
    return p, blocks, r


def test_block_formula_equals_brute_force(tiny):
    p, blocks, r = tiny
    ns, nt = p.ns, p.nt
    Phi_s, T = r["Phi_s"], r["T"]
    mu = np.array([1.1, 0.4])
    A = fom.affine_operator(p.rowptr, p.col, p.vals, p.theta(mu))
    Ast, fst = fom.st_fom_system(A, p.dt, p.B, p.F, p.u0)
    Pst = strom.st_basis(Phi_s, T, ns, nt)
    brute = Pst.T @ (Ast @ Pst)
    rm = strom.ReducedModel(p, Phi_s, T, ns, nt)
    blockf = strom.st_operator(rm.Ahat(p.theta(mu)), rm.G, rm.M, rm.S, ns, nt)
    literal = strom.st_operator_literal(rm.Ahat(p.theta(mu)), T, p.dt, ns, nt)
    sc = np.abs(brute).max()
    assert np.abs(blockf - brute).max() < 1e-13 * sc
    assert np.abs(literal - brute).max() < 1e-13 * sc
    # reduced input and initial vectors (Eqs. j-block-vector, ststate)
    f_only = np.concatenate([p.dt[k] * (p.B @ p.F[k]) for k in range(p.Nt)])
    u0st = np.zeros(p.N * p.Nt)
    u0st[:p.N] = p.u0
    assert np.abs(rm.fhat - Pst.T @ f_only).max() < 1e-14 * np.abs(rm.fhat).max()
    assert np.abs(rm.u0hat - Pst.T @ u0st).max() < 1e-14 * np.abs(rm.u0hat).max()
    # the printed initial-vector formula does not equal Phi_st^T u0^st here
    printed = strom.st_initial_printed(Phi_s, T, p.u0, ns, nt)
    assert np.abs(printed - Pst.T @ u0st).max() > 1e-3 * np.abs(rm.u0hat).max()


def test_spacetime_basis_orthonormal(tiny):
    p, blocks, r = tiny
    Pst = strom.st_basis(r["Phi_s"], r["T"], p.ns, p.nt)
    assert np.abs(Pst.T @ Pst - np.eye(p.ns * p.nt)).max() < 1e-13
    # reconstruction by blocks equals Phi_st uhat (Eq. ststateapproximation)
    uh = np.random.default_rng(1).standard_normal(p.ns * p.nt)
    U = strom.reconstruct(r["Phi_s"], r["T"], uh, p.ns, p.ns, p.nt)
    assert np.abs(U.T.reshape(-1) - Pst @ uh).max() < 1e-14


def test_full_bases_reproduce_fom(tiny):
    # Complete Phi_s (N x N) and each Phi_t^i (Nt x Nt) to square orthogonal
    # matrices: the space-time Galerkin system is then A^st itself in another
    # basis, so the ROM equals the FOM at any parameter.
    p, blocks, r = tiny
    rng = np.random.default_rng(3)
    N, Nt = p.N, p.Nt
    Phi = np.linalg.qr(np.concatenate([r["Phi_s"], rng.standard_normal((N, N - p.ns))], 1))[0]
    T = np.zeros((Nt, N * Nt))
    for i in range(N):
        if i < p.ns:
            seed = r["T"][:, [i + p.ns * j for j in range(p.nt)]]
        else:
            seed = np.zeros((Nt, 0))
        Ti = np.linalg.qr(np.concatenate([seed, rng.standard_normal((Nt, Nt - seed.shape[1]))], 1))[0]
        for j in range(Nt):
            T[:, i + N * j] = Ti[:, j]
    rm = strom.ReducedModel(p, Phi, T, N, Nt)
    for mu in p.test_mu[:2]:
        A = fom.affine_operator(p.rowptr, p.col, p.vals, p.theta(mu))
        Uf = fom.fom_march(A, p.dt, p.B, p.F, p.u0)
        Ur = rm.reconstruct(rm.solve(p.theta(mu)))
        assert strom.rel_error(Uf, Ur) < 1e-11


def test_untruncated_reproduces_training_solutions(tiny):
    # With ns = rank U and nt = rank Upsilon_i the training solutions lie in
    # range(Phi_st), so the Galerkin ROM reproduces them exactly.
    p, blocks, r = tiny
    U = pod.snapshot_matrix(blocks)
    rank = np.linalg.matrix_rank(U, tol=1e-12 * np.linalg.norm(U, 2))
    n_mu = len(blocks)
    r2 = pod.pod_exact(blocks, rank, n_mu)
    rm = strom.ReducedModel(p, r2["Phi_s"], r2["T"], rank, n_mu)
    for k, mu in enumerate(p.train_mu):
        Ur = rm.reconstruct(rm.solve(p.theta(mu)))
        assert strom.rel_error(blocks[k], Ur) < 1e-9


def test_nested_truncation_is_principal_submatrix(tiny):
    p, blocks, r = tiny
    ns_m, nt_m = 2, 2
    rm = strom.ReducedModel(p, r["Phi_s"], r["T"], p.ns, p.nt)
    th = p.theta(np.array([0.7, 0.5]))
    A_sub, f_sub = rm.operator(th, ns_m, nt_m)
    # build the (2, 2) model from truncated bases directly
    T2 = np.zeros((p.Nt, ns_m * nt_m))
    for i in range(ns_m):
        for j in range(nt_m):
            T2[:, i + ns_m * j] = r["T"][:, i + p.ns * j]
    rm2 = strom.ReducedModel(p, r["Phi_s"][:, :ns_m], T2, ns_m, nt_m)
    A2, f2 = rm2.operator(th)
    assert np.abs(A_sub - A2).max() < 1e-13 * np.abs(A2).max()
    assert np.abs(f_sub - f2).max() < 1e-13 * np.abs(f2).max()


def test_theorem3_error_bound(tiny):
    # ||du^st||_inf <= sqrt(Nt) ||(A^st)^-1||_2 ||r^st(u~)||_inf (Thm. 3).
    p, blocks, r = tiny
    rm = strom.ReducedModel(p, r["Phi_s"], r["T"], p.ns, p.nt)
    for mu in p.test_mu:
        A = fom.affine_operator(p.rowptr, p.col, p.vals, p.theta(mu))
        Ast, rhs = fom.st_fom_system(A, p.dt, p.B, p.F, p.u0)
        Uf = fom.fom_march(A, p.dt, p.B, p.F, p.u0)
        Ur = rm.reconstruct(rm.solve(p.theta(mu)))
        ust = Ur.T.reshape(-1)
        res = (Ast @ ust - rhs).reshape(p.Nt, p.N).T
        smin = sla.svdvals(Ast.toarray()).min()
        lhs = strom.st_inf_norm(Uf - Ur)
        bound = np.sqrt(p.Nt) / smin * strom.st_inf_norm(res)
        assert lhs <= bound * (1 + 1e-12)


# ---- spatial Galerkin ROM (Sec. 3.1) and its error bound (Theorem 1) ----------

def _ragged_dt(p):
    # non-uniform steps, so that a step index off by one changes the result
    return p.dt * (1.0 + 0.5 * np.sin(np.arange(p.Nt) + 1.0))


def test_spatial_rom_full_basis_reproduces_fom(tiny):
    # a square orthogonal Phi_s makes Eq. space_reduced_discretized_ODE the
    # FOM (Eq. fom) in another basis, at any step sizes
    p, blocks, r = tiny
    rng = np.random.default_rng(4)
    Phi = np.linalg.qr(np.concatenate([r["Phi_s"], rng.standard_normal((p.N, p.N - p.ns))], 1))[0]
    Ahat_q = strom.spatial_reduced(p.rowptr, p.col, p.vals, Phi)
    dt = _ragged_dt(p)
    for mu in p.test_mu[:2]:
        th = p.theta(mu)
        A = fom.affine_operator(p.rowptr, p.col, p.vals, th)
        Uf = fom.fom_march(A, dt, p.B, p.F, p.u0, solver="dense")
        Uh = strom.spatial_march(np.tensordot(th, Ahat_q, axes=(0, 0)), Phi.T @ p.B, p.F, dt,
                                 Phi.T @ p.u0)
        assert strom.rel_error(Uf, Phi @ Uh) < 1e-12


def test_spatial_rom_residual_orthogonal_to_basis(tiny):
    # the ROM state u~^k = Phi_s uhat^k leaves a full-order residual (Eq.
    # residual) that is nonzero but orthogonal to range(Phi_s) (Eq. approxres)
    p, blocks, r = tiny
    Phi = r["Phi_s"]
    Ahat_q = strom.spatial_reduced(p.rowptr, p.col, p.vals, Phi)
    dt = _ragged_dt(p)
    for mu in p.test_mu[:3]:
        th = p.theta(mu)
        A = fom.affine_operator(p.rowptr, p.col, p.vals, th)
        Uh = strom.spatial_march(np.tensordot(th, Ahat_q, axes=(0, 0)), Phi.T @ p.B, p.F, dt,
                                 Phi.T @ p.u0)
        Ut = Phi @ Uh
        R = strom.fom_residual(A, dt, p.B, p.F, Ut, Phi @ (Phi.T @ p.u0))
        scale = np.abs(Ut).max()
        assert np.abs(R).max() > 1e-6 * scale
        assert np.abs(Phi.T @ R).max() < 1e-13 * scale


def test_spatial_rom_equals_spacetime_rom_with_complete_temporal_bases(tiny):
    # with every Phi_t^i completed to an Nt x Nt orthogonal matrix, range(Phi_st)
    # = range(I_Nt (x) Phi_s): the space-time Galerkin solution (Eq.
    # st-galerkin) is then the spatial ROM trajectory, also for nested ns
    p, blocks, r = tiny
    ns, Nt = p.ns, p.Nt
    rng = np.random.default_rng(5)
    T = np.zeros((Nt, ns * Nt))
    for i in range(ns):
        seed = r["T"][:, [i + ns * j for j in range(p.nt)]]
        Ti = np.linalg.qr(np.concatenate([seed, rng.standard_normal((Nt, Nt - p.nt))], 1))[0]
        for j in range(Nt):
            T[:, i + ns * j] = Ti[:, j]
    rm = strom.ReducedModel(p, r["Phi_s"], T, ns, Nt)
    for mu in p.test_mu[:3]:
        th = p.theta(mu)
        for ns_m in (ns, 2):
            Ust = rm.reconstruct(rm.solve(th, ns_m, Nt), ns_m, Nt)
            Usp = r["Phi_s"][:, :ns_m] @ rm.spatial_march(th, ns_m)
            assert strom.rel_error(Usp, Ust) < 1e-12


def test_theorem1_error_bound(tiny):
    # ||u^k - u~^k|| <= sum_{i<=k} prod_{j=i..k} xi_j ||r^i|| (Theorem 1), from
    # the one-step identity e^k = (I - dt_k A)^-1 (e^{k-1} - r^k) (Eq. rearrange)
    p, blocks, r = tiny
    rm = strom.ReducedModel(p, r["Phi_s"], r["T"], p.ns, p.nt)
    Phi = r["Phi_s"]
    for mu in p.test_mu:
        th = p.theta(mu)
        A = fom.affine_operator(p.rowptr, p.col, p.vals, th)
        Uf = fom.fom_march(A, p.dt, p.B, p.F, p.u0, solver="dense")
        Ut = Phi @ rm.spatial_march(th)
        ut0 = Phi @ rm.u0s
        R = strom.fom_residual(A, p.dt, p.B, p.F, Ut, ut0)
        E = Uf - Ut
        e = p.u0 - ut0
        scale = np.abs(Uf).max()
        for k in range(p.Nt):
            step = np.linalg.solve(np.eye(p.N) - p.dt[k] * A.toarray(), e - R[:, k])
            assert np.abs(E[:, k] - step).max() < 1e-12 * scale
            e = E[:, k]
        bound = strom.spatial_error_bound(A, p.dt, R, float(np.linalg.norm(p.u0 - ut0)))
        err = np.linalg.norm(E, axis=0)
        assert err.max() > 1e-8 * scale
        assert (err <= bound * (1 + 1e-12)).all()


def test_theorem1_bound_is_attained_for_aligned_scalar_errors():
    # N = 1, A = a < 0: xi_k = 1 / (1 - dt_k a) > 0 and e^k = xi_k (e^{k-1} -
    # r^k).  With e^0 >= 0 and every r^k <= 0 no term cancels, so the triangle
    # inequalities of the proof are equalities and the bound equals |e^k|.
    a = -2.0
    dt = np.array([0.1, 0.3, 0.05, 0.2, 0.15])
    A = np.array([[a]])
    B = np.array([[1.0]])
    F = np.array([[1.0], [0.5], [-2.0], [0.0], [3.0]])
    u0 = np.array([0.7])
    U = fom.fom_march(sp.csr_matrix(A), dt, B, F, u0, solver="dense")
    c = np.array([0.3, 0.01, 0.2, 0.05, 0.4])   # r^k = -c_k
    e0 = 0.25
    E = np.empty(len(dt))
    e = e0
    for k in range(len(dt)):
        e = (e + c[k]) / (1.0 - dt[k] * a)
        E[k] = e
    Ut = U - E[None, :]
    R = strom.fom_residual(A, dt, B, F, Ut, u0 - e0)
    assert np.abs(R[0] + c).max() < 1e-14
    bound = strom.spatial_error_bound(A, dt, R, e0)
    assert np.abs(bound - E).max() < 1e-14 * E.max()
