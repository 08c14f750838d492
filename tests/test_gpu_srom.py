"""GPU parity of the batched spatial Galerkin ROM (Sec. 3.1, Eq.
space_reduced_discretized_ODE) against the oracle, through the C ABI.

Tolerance: the kernel inverts I - dt Ahat(mu) once by Gauss-Jordan with
partial pivoting and multiplies; the oracle solves each step by LAPACK.  Both
are backward stable, the matrices are well conditioned (cond < 1e2 here) and
the march contracts errors, so after Nt steps the two trajectories differ by
a few hundred ulps of max |uhat| at most: 1e-11 relative."""
import numpy as np
import pytest

from gpu_util import dev_B, dev_tensor, make_model, oracle_fom, rel_max
from oracle import fom, pod, strom
from workloads import make_problem, problem_for

pytestmark = pytest.mark.gpu


def _torch():
    return __import__("torch")


@pytest.fixture(scope="module")
def c1_model():
    p = problem_for("c1")
    blocks = oracle_fom(p, p.train_mu)
    ref = pod.pod_exact(blocks, p.ns, p.nt)
    return p, ref, strom.ReducedModel(p, ref["Phi_s"], ref["T"], p.ns, p.nt)


def _gpu_model(p, Phi, T, ns, nt, dt=None, u0=None):
    m = make_model(p)
    m.st_model_set_basis(ns, nt, p.Nt, dev_tensor(Phi.T.copy()), dev_tensor(T.T.copy()))
    m.st_rom_assemble(p.dt if dt is None else dt, dev_B(p), p.F, None if u0 is None else dev_tensor(u0))
    return m


def _march(m, thetas, sizes, Nt, ns):
    torch = _torch()
    n = len(thetas)
    sz = None if sizes is None else dev_tensor(np.asarray(sizes, dtype=np.int32))
    u = torch.full((n, Nt, ns), float("nan"), dtype=torch.float64, device="cuda:0")
    status = torch.full((n,), -1, dtype=torch.int32, device="cuda:0")
    m.st_rom_spatial_march(n, dev_tensor(np.asarray(thetas)), sz, u, status)
    torch.cuda.synchronize()
    return u.cpu().numpy(), status.cpu().numpy()


def test_spatial_march_uneven_sizes(c1_model):
    p, ref, rm = c1_model
    m = _gpu_model(p, ref["Phi_s"], ref["T"], p.ns, p.nt)
    rng = np.random.default_rng(21)
    n = 200
    mus = p.mu_lo + rng.random((n, 2)) * (p.mu_hi - p.mu_lo)
    sizes = rng.choice([1, 2, 5, 7, 8], size=n).astype(np.int32)
    U, status = _march(m, p.theta(mus), sizes, p.Nt, p.ns)
    assert (status == 0).all()
    for k in range(n):
        a = sizes[k]
        want = rm.spatial_march(p.theta(mus[k]), a)
        assert rel_max(U[k, :, :a].T, want) < 1e-11
        assert np.isnan(U[k, :, a:]).all()  # entries past ns_p are left alone
    m.close()


def test_spatial_march_ragged_steps_and_initial_state():
    # 2-D S4 case, u0 != 0, non-uniform steps: one inverse per distinct step
    p = make_problem(dim=2, M=8, quad="s4", Nt=9, u0="seeded", g="sin", source="gaussian",
                     ns=5, nt=3)
    blocks = oracle_fom(p, p.train_mu, u0=p.u0)
    ref = pod.pod_exact(blocks, p.ns, p.nt)
    rm = strom.ReducedModel(p, ref["Phi_s"], ref["T"], p.ns, p.nt)
    dt = p.dt * np.array([1.0, 1.0, 0.5, 0.5, 2.0, 1.0, 1.0, 0.25, 0.75])
    m = _gpu_model(p, ref["Phi_s"], ref["T"], p.ns, p.nt, dt=dt, u0=p.u0)
    assert np.abs(rm.u0s).max() > 1e-3
    mus = p.test_mu
    sizes = np.array([5, 3, 1, 4, 5, 2, 5, 5][:len(mus)], dtype=np.int32)
    U, status = _march(m, p.theta(mus), sizes, p.Nt, p.ns)
    assert (status == 0).all()
    for k, mu in enumerate(mus):
        a = sizes[k]
        want = strom.spatial_march(rm.Ahat(p.theta(mu))[:a, :a], rm.Bhat[:a], p.F, dt, rm.u0s[:a])
        assert rel_max(U[k, :, :a].T, want) < 1e-11
    m.close()


def test_spatial_march_full_basis_reproduces_fom():
    # a square orthogonal Phi_s: the spatial ROM is the FOM in another basis
    p = make_problem(dim=1, M=8, quad="gl4", Nt=6, u0="seeded", g="sin", ns=4, nt=1)
    N = p.N
    Phi = np.linalg.qr(np.random.default_rng(8).standard_normal((N, N)))[0]
    T = np.zeros((p.Nt, N))
    T[0] = 1.0                       # any unit temporal columns (unused here)
    m = _gpu_model(p, Phi, T, N, 1, u0=p.u0)
    U, status = _march(m, p.theta(p.test_mu), None, p.Nt, N)
    assert (status == 0).all()
    for k, mu in enumerate(p.test_mu):
        A = fom.affine_operator(p.rowptr, p.col, p.vals, p.theta(mu))
        Uf = fom.fom_march(A, p.dt, p.B, p.F, p.u0, solver="dense")
        assert strom.rel_error(Uf, Phi @ U[k].T) < 1e-12
    m.close()


def test_spatial_march_wide_basis():
    # ns above the block's 128 threads: one part per row, rows strided
    p = problem_for("c1")
    ns = 130
    Phi = np.linalg.qr(np.random.default_rng(12).standard_normal((p.N, ns)))[0]
    T = np.zeros((p.Nt, ns))
    T[0] = 1.0
    m = _gpu_model(p, Phi, T, ns, 1)
    Ahat_q = strom.spatial_reduced(p.rowptr, p.col, p.vals, Phi)
    Bhat = Phi.T @ p.B
    mus = p.test_mu[:3]
    sizes = np.array([130, 129, 64], dtype=np.int32)
    U, status = _march(m, p.theta(mus), sizes, p.Nt, ns)
    assert (status == 0).all()
    for k, mu in enumerate(mus):
        a = sizes[k]
        Ah = np.tensordot(p.theta(mu), Ahat_q, axes=(0, 0))[:a, :a]
        want = strom.spatial_march(Ah, Bhat[:a], p.F, p.dt)
        assert rel_max(U[k, :, :a].T, want) < 1e-11
    m.close()


def test_spatial_march_equals_spacetime_solve_with_complete_temporal_bases(c1_model):
    # with every Phi_t^i completed to Nt x Nt the space-time ROM (st_rom_solve)
    # and the spatial ROM give the same trajectory
    torch = _torch()
    p, ref, rm = c1_model
    ns, Nt = p.ns, p.Nt
    rng = np.random.default_rng(9)
    T = np.zeros((Nt, ns * Nt))
    for i in range(ns):
        seed = ref["T"][:, [i + ns * j for j in range(p.nt)]]
        Ti = np.linalg.qr(np.concatenate([seed, rng.standard_normal((Nt, Nt - p.nt))], 1))[0]
        for j in range(Nt):
            T[:, i + ns * j] = Ti[:, j]
    m = _gpu_model(p, ref["Phi_s"], T, ns, Nt)
    th = p.theta(p.test_mu[:4])
    U, status = _march(m, th, None, Nt, ns)
    assert (status == 0).all()
    n = len(th)
    uh = torch.zeros((n, ns * Nt), dtype=torch.float64, device="cuda:0")
    st_status = torch.full((n,), -1, dtype=torch.int32, device="cuda:0")
    m.st_rom_solve(n, dev_tensor(th), None, uh, None, st_status)
    torch.cuda.synchronize()
    assert (st_status.cpu().numpy() == 0).all()
    uh = uh.cpu().numpy()
    for k in range(n):
        C = np.zeros((ns, Nt))                      # C[i, k] = sum_j uhat_ij phi_t^{ij}[k]
        for i in range(ns):
            for j in range(Nt):
                C[i] += uh[k, i + ns * j] * T[:, i + ns * j]
        assert rel_max(U[k].T, C) < 1e-10
    m.close()


def test_spatial_march_status_codes(c1_model):
    import paper_1910_01260_gb300 as st
    p, ref, rm = c1_model
    m = _gpu_model(p, ref["Phi_s"], ref["T"], p.ns, p.nt)
    th = p.theta(p.test_mu[:4]).copy()
    th[1, 0] = np.nan                    # a non-finite pivot column: singular
    U, status = _march(m, th, [8, 8, 0, 9], p.Nt, p.ns)
    assert status[0] == st.ST_OK
    assert status[1] == st.ST_ERR_SINGULAR and np.isnan(U[1]).all()
    assert status[2] == st.ST_ERR_ARG and status[3] == st.ST_ERR_ARG
    with pytest.raises(st.StError):
        m.st_sync()
    # the model stays usable
    U2, status2 = _march(m, th[:1], None, p.Nt, p.ns)
    assert status2[0] == st.ST_OK and np.array_equal(U2[0], U[0])
    m.close()


def test_spatial_march_independent_of_batching(c1_model):
    p, ref, rm = c1_model
    m = _gpu_model(p, ref["Phi_s"], ref["T"], p.ns, p.nt)
    th = p.theta(p.test_mu)
    full, _ = _march(m, th, None, p.Nt, p.ns)
    for k in range(len(th)):
        one, _ = _march(m, th[k:k + 1], None, p.Nt, p.ns)
        assert np.array_equal(one[0], full[k])
    m.close()


def test_spatial_march_requires_assembly():
    import paper_1910_01260_gb300 as st
    p = make_problem(dim=1, M=8, quad="gl4", Nt=6, ns=3, nt=2)
    m = make_model(p)
    with pytest.raises(st.StError) as e:
        _march(m, p.theta(p.test_mu[:1]), None, p.Nt, 3)
    assert e.value.code == st.ST_ERR_STATE
    m.close()
