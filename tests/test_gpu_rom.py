"""GPU parity of assembly (Sec. 4.3), batched reduced solve (Eq. st-galerkin)
and reconstruction against the oracle, given the oracle's bases.

Tolerances: assembly is a fixed sequence of FP64 sums, 1e-12 relative; the
reduced solve is LAPACK-equivalent partial-pivot LU plus one refinement step,
so the solution error is bounded by ~n eps cond(Ahat^st) (cond <= 1e3 here):
1e-10 relative; reconstruction is a short FP64 contraction, 1e-13."""
import numpy as np
import pytest

from gpu_util import dev_B, dev_tensor, make_model, oracle_fom, rel_max
from oracle import pod, strom
from workloads import make_problem, problem_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c1_model():
    p = problem_for("c1")
    blocks = oracle_fom(p, p.train_mu)
    ref = pod.pod_exact(blocks, p.ns, p.nt)
    return p, ref, strom.ReducedModel(p, ref["Phi_s"], ref["T"], p.ns, p.nt)


def _gpu_model(p, ref, ns, nt, u0=None, **opts):
    m = make_model(p, **opts)
    m.st_model_set_basis(ns, nt, p.Nt, dev_tensor(ref["Phi_s"].T.copy()), dev_tensor(ref["T"].T.copy()))
    m.st_rom_assemble(p.dt, dev_B(p), p.F, None if u0 is None else dev_tensor(u0))
    return m


def test_assembly_matches_block_formulas(c1_model):
    p, ref, rm = c1_model
    m = _gpu_model(p, ref, p.ns, p.nt)
    Ahat, G, M, S, rhs = m.st_model_get_reduced(p.ns, p.nt)
    assert rel_max(Ahat, rm.Ahat_q) < 1e-12
    assert rel_max(G, rm.G) < 1e-12
    assert rel_max(M, rm.M) < 1e-12
    assert rel_max(S, rm.S) < 1e-12
    assert rel_max(rhs, rm.fhat + rm.u0hat) < 1e-12
    m.close()


def test_assembly_with_initial_state():
    p = make_problem(dim=2, M=8, quad="s4", Nt=9, u0="seeded", g="sin", source="gaussian",
                     ns=5, nt=3)
    blocks = oracle_fom(p, p.train_mu, u0=p.u0)
    ref = pod.pod_exact(blocks, p.ns, p.nt)
    rm = strom.ReducedModel(p, ref["Phi_s"], ref["T"], p.ns, p.nt)
    m = _gpu_model(p, ref, p.ns, p.nt, u0=p.u0)
    Ahat, G, M, S, rhs = m.st_model_get_reduced(p.ns, p.nt)
    assert np.abs(rm.u0hat).max() > 1e-3
    assert rel_max(rhs, rm.fhat + rm.u0hat) < 1e-12
    m.close()


def _solve(m, thetas, sizes, n_full):
    torch = __import__("torch")
    n = len(thetas)
    th = dev_tensor(thetas)
    sz = None if sizes is None else dev_tensor(np.asarray(sizes, dtype=np.int32))
    uhat = torch.full((n, n_full), float("nan"), dtype=torch.float64, device="cuda:0")
    res = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    status = torch.full((n,), -1, dtype=torch.int32, device="cuda:0")
    m.st_rom_solve(n, th, sz, uhat, res, status)
    torch.cuda.synchronize()
    return uhat.cpu().numpy(), res.cpu().numpy(), status.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_batched_solve_uneven_sizes(c1_model, precision):
    # precision 1: FP32 assembly; 2: FP32 assembly and LU factors.  The FP64
    # residual refinement brings both back to the FP64 tolerance.
    p, ref, rm = c1_model
    m = _gpu_model(p, ref, p.ns, p.nt, precision=precision, refine_steps=(1, 2, 3)[precision])
    rng = np.random.default_rng(11)
    n = 300
    mus = p.mu_lo + rng.random((n, 2)) * (p.mu_hi - p.mu_lo)
    choices = np.array([(8, 4), (4, 2), (6, 3), (1, 1), (8, 1), (3, 4)], dtype=np.int32)
    sizes = choices[rng.integers(0, len(choices), n)]
    uh, res, status = _solve(m, p.theta(mus), sizes, p.ns * p.nt)
    assert (status == 0).all()
    assert res.max() < 1e-12
    for k in range(n):
        a, b = sizes[k]
        want = rm.solve(p.theta(mus[k]), a, b)
        assert rel_max(uh[k, :a * b], want) < 1e-10
    m.close()


def test_solve_batch_independent_of_batching(c1_model):
    p, ref, rm = c1_model
    m = _gpu_model(p, ref, p.ns, p.nt)
    mus = p.test_mu
    th = p.theta(mus)
    full, _, _ = _solve(m, th, None, p.ns * p.nt)
    for k in range(len(mus)):
        one, _, _ = _solve(m, th[k:k + 1], None, p.ns * p.nt)
        assert np.array_equal(one[0], full[k])
    m.close()


def test_solve_reports_singular_and_bad_sizes():
    import paper_1910_01260_gb300 as st
    p = make_problem(dim=1, M=8, quad="gl4", Nt=6, ns=3, nt=2)
    m = make_model(p)
    z = dev_tensor(np.zeros((3, p.N)))
    zt = dev_tensor(np.zeros((6, p.Nt)))
    m.st_model_set_basis(3, 2, p.Nt, z, zt)
    m.st_rom_assemble(p.dt, dev_B(p), p.F, None)
    uh, res, status = _solve(m, p.theta(p.train_mu[:2]), [(3, 2), (4, 2)], 6)
    assert status[0] == st.ST_ERR_SINGULAR
    assert status[1] == st.ST_ERR_ARG
    with pytest.raises(st.StError):
        m.st_sync()
    m.close()


def test_reconstruction_and_outputs(c1_model):
    torch = __import__("torch")
    p, ref, rm = c1_model
    m = _gpu_model(p, ref, p.ns, p.nt)
    rng = np.random.default_rng(5)
    n = 5
    sizes = np.array([(8, 4), (3, 2), (8, 1), (1, 4), (5, 3)], dtype=np.int32)
    nf = p.ns * p.nt
    uh = np.zeros((n, nf))
    for k, (a, b) in enumerate(sizes):
        uh[k, :a * b] = rng.standard_normal(a * b)
    u = torch.zeros((n, p.Nt, p.N), dtype=torch.float64, device="cuda:0")
    Cout = rng.standard_normal((p.N, 3))
    y = torch.zeros((n, p.Nt, 3), dtype=torch.float64, device="cuda:0")
    m.st_rom_reconstruct(n, dev_tensor(uh), dev_tensor(sizes), u, 3, dev_tensor(Cout.T.copy()), y)
    torch.cuda.synchronize()
    U = u.cpu().numpy()
    Y = y.cpu().numpy()
    for k, (a, b) in enumerate(sizes):
        want = strom.reconstruct(ref["Phi_s"], ref["T"], uh[k, :a * b], p.ns, a, b)
        assert rel_max(U[k].T, want) < 1e-13
        assert rel_max(Y[k].T, Cout.T @ want) < 1e-12
    m.close()


def test_set_options_switches_precision(c1_model):
    import paper_1910_01260_gb300 as st
    p, ref, rm = c1_model
    m = _gpu_model(p, ref, p.ns, p.nt)
    th = p.theta(p.test_mu)
    a, _, _ = _solve(m, th, None, p.ns * p.nt)
    m.st_model_set_options(precision=st.ST_FP32_LU, refine_steps=3)
    b, res, status = _solve(m, th, None, p.ns * p.nt)
    assert (status == 0).all() and res.max() < 1e-12
    assert rel_max(b, a) < 1e-10
    with pytest.raises(st.StError):
        m.st_model_set_options(precision=7)
    m.close()
