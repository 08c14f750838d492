"""Reduced solves by preconditioned Richardson refinement (reference inverses
of Ahat^st at the training parameters), started from the surrogate or from
zero: the answers meet the gate on the oracle's own FP64 residual and match
the oracle's LAPACK solutions; the surrogate start needs no more corrections
than the zero start; samples left above the gate get the batched LU."""
import numpy as np
import pytest

from gpu_util import dev_B, dev_tensor, make_model, oracle_fom
from oracle import pod, strom
from workloads import problem_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c1_setup():
    p = problem_for("c1")
    blocks = oracle_fom(p, p.train_mu)
    ref = pod.pod_block_incremental(blocks, p.ns, p.nt, r_max=200)
    return p, ref


def _model(p, ref):
    m = make_model(p)
    m.st_model_set_basis(p.ns, p.nt, p.Nt, dev_tensor(ref["Phi_s"].T.copy()), dev_tensor(ref["T"].T.copy()))
    m.st_rom_assemble(p.dt, dev_B(p), p.F, None)
    m.st_rom_precond_build(p.train_mu, p.theta(p.train_mu))
    return m


def _batch(p, n, seed=4):
    rng = np.random.default_rng(seed)
    return p.mu_lo + rng.random((n, 2)) * (p.mu_hi - p.mu_lo)


def _refine(m, p, mu, guess, gate, max_iter):
    torch = __import__("torch")
    n, nf = len(mu), p.ns * p.nt
    uh = torch.zeros((n, nf), dtype=torch.float64, device="cuda:0")
    rr = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    used = torch.zeros(n, dtype=torch.int32, device="cuda:0")
    it, nfb = m.st_rom_refine(n, dev_tensor(mu), dev_tensor(p.theta(mu)), guess, gate, max_iter, uh, rr, used)
    m.st_sync()
    return uh.cpu().numpy(), rr.cpu().numpy(), used.cpu().numpy(), it, nfb


def test_refinement_meets_the_gate_on_the_oracle_residual(c1_setup):
    import paper_1910_01260_gb300 as st
    p, ref = c1_setup
    m = _model(p, ref)
    rm = strom.ReducedModel(p, ref["Phi_s"], ref["T"], p.ns, p.nt)
    mu = _batch(p, 300)
    gate = 1e-6
    U, rel, used, it, nfb = _refine(m, p, mu, st.ST_GUESS_ZERO, gate, 50)
    assert nfb == 0 and (used == 0).all() and 1 <= it <= 50
    for k in range(0, 300, 7):
        A, f = rm.operator(p.theta(mu[k]))
        r_oracle = np.linalg.norm(f - A @ U[k]) / np.linalg.norm(f)
        # the library's residual uses FP32-accurate products (tensor-core FP32
        # sums of three-part BF16 splits): a few 1e-7 of ||rhs|| here
        assert r_oracle <= gate * (1 + 1e-2) + 5e-7
        assert abs(r_oracle - rel[k]) <= 5e-7 + 1e-2 * r_oracle
        want = np.linalg.solve(A, f)
        assert np.linalg.norm(U[k] - want) / np.linalg.norm(want) <= 100 * gate
    m.close()


def test_surrogate_start_saves_corrections(c1_setup):
    torch = __import__("torch")
    import paper_1910_01260_gb300 as st
    p, ref = c1_setup
    m = _model(p, ref)
    mu_tr = _batch(p, 2048, seed=5)
    u_tr = torch.zeros((2048, p.ns * p.nt), dtype=torch.float64, device="cuda:0")
    m.st_rom_solve(2048, dev_tensor(p.theta(mu_tr)), None, u_tr)
    m.st_rom_surrogate_train(2048, dev_tensor(mu_tr), p.mu_lo, p.mu_hi, u_tr, epochs=60, batch=256, lr=2e-3)
    mu = _batch(p, 500, seed=6)
    its = {}
    for guess in (st.ST_GUESS_ZERO, st.ST_GUESS_SURROGATE):
        U, rel, used, it, nfb = _refine(m, p, mu, guess, 1e-6, 50)
        assert nfb == 0 and rel.max() <= 1e-6
        its[guess] = it
    assert its[st.ST_GUESS_SURROGATE] <= its[st.ST_GUESS_ZERO]
    m.close()


def test_samples_above_the_gate_fall_back_to_the_lu(c1_setup):
    torch = __import__("torch")
    import paper_1910_01260_gb300 as st
    p, ref = c1_setup
    m = _model(p, ref)
    mu = _batch(p, 64)
    U, rel, used, it, nfb = _refine(m, p, mu, st.ST_GUESS_ZERO, 0.0, 1)    # gate 0: nobody passes
    assert it == 1 and nfb == 64 and (used == 1).all()
    lu = torch.zeros((64, p.ns * p.nt), dtype=torch.float64, device="cuda:0")
    lr = torch.zeros(64, dtype=torch.float64, device="cuda:0")
    m.st_rom_solve(64, dev_tensor(p.theta(mu)), None, lu, lr)
    m.st_sync()
    assert np.array_equal(U, lu.cpu().numpy()) and np.array_equal(rel, lr.cpu().numpy())
    m.close()


def test_refine_needs_a_preconditioner(c1_setup):
    import paper_1910_01260_gb300 as st
    p, ref = c1_setup
    m = make_model(p)
    m.st_model_set_basis(p.ns, p.nt, p.Nt, dev_tensor(ref["Phi_s"].T.copy()), dev_tensor(ref["T"].T.copy()))
    m.st_rom_assemble(p.dt, dev_B(p), p.F, None)
    with pytest.raises(st.StError) as e:
        _refine(m, p, _batch(p, 4), st.ST_GUESS_ZERO, 1e-6, 5)
    assert e.value.code == st.ST_ERR_STATE
    m.close()
