"""Persistence and resumable basis builds on the GPU: a model saved and
loaded solves bit for bit like the original, and an incremental SVD fed in
two sittings (save and load between them) equals one fed all at once."""
import numpy as np
import pytest

from gpu_util import dev_B, dev_tensor, make_model, oracle_fom
from oracle import pod
from workloads import problem_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c1():
    p = problem_for("c1")
    return p, oracle_fom(p, p.train_mu)


def _snaps(blocks):
    return dev_tensor(np.stack([b.T for b in blocks]))  # column p*Nt + k


def _solve(m, p, mu):
    torch = __import__("torch")
    n = p.ns * p.nt
    uh = torch.zeros((len(mu), n), dtype=torch.float64, device="cuda:0")
    rr = torch.zeros(len(mu), dtype=torch.float64, device="cuda:0")
    m.st_rom_solve(len(mu), dev_tensor(p.theta(mu)), None, uh, rr)
    m.st_sync()
    return uh.cpu().numpy(), rr.cpu().numpy()


def test_save_load_round_trip(c1, tmp_path):
    torch = __import__("torch")
    import paper_1910_01260_gb300 as st
    p, blocks = c1
    m = make_model(p, r_max=200, precision=st.ST_FP32_LU, refine_steps=2)
    m.st_rom_build_basis(len(blocks), p.Nt, _snaps(blocks), p.ns, p.nt)
    m.st_rom_assemble(p.dt, dev_B(p), p.F, None)
    mu = p.test_mu
    u_a, r_a = _solve(m, p, mu)
    # a briefly trained surrogate travels with the model
    mu_tr = np.asarray(p.train_mu, dtype=np.float64)
    mu_tr = np.concatenate([mu_tr, np.asarray(mu, dtype=np.float64)])
    u_tr = torch.zeros((len(mu_tr), p.ns * p.nt), dtype=torch.float64, device="cuda:0")
    m.st_rom_solve(len(mu_tr), dev_tensor(p.theta(mu_tr)), None, u_tr)
    m.st_rom_surrogate_train(len(mu_tr), dev_tensor(mu_tr), p.mu_lo, p.mu_hi, u_tr, epochs=3, batch=4)
    path = tmp_path / "c1.strom"
    m.st_model_save(str(path))
    info = st.st_model_file_info(str(path))
    assert (info["n_rows"], info["ns"], info["nt"], info["Nt"]) == (p.N, p.ns, p.nt, p.Nt)
    assert info["assembled"] == 1 and info["surrogate"] == 1 and info["pod_rank"] > 0
    m2 = st.Model.st_model_load(str(path), stream=torch.cuda.current_stream().cuda_stream)
    assert m2.opts.precision == st.ST_FP32_LU and m2.opts.refine_steps == 2
    u_b, r_b = _solve(m2, p, mu)
    assert np.array_equal(u_a, u_b) and np.array_equal(r_a, r_b)
    # operators, bases, incremental-SVD state and surrogate are the saved ones
    for a, b in zip(m.st_model_get_reduced(p.ns, p.nt), m2.st_model_get_reduced(p.ns, p.nt)):
        assert np.array_equal(a, b)
    sa, ra = m.st_pod_get_state()
    sb, rb = m2.st_pod_get_state()
    assert ra == rb and np.array_equal(sa, sb)
    assert m.st_pod_get_stats() == m2.st_pod_get_stats()
    assert np.array_equal(m.st_rom_surrogate_params(), m2.st_rom_surrogate_params())
    n = len(mu)
    outs = []
    for mm in (m, m2):
        uh = torch.zeros((n, p.ns * p.nt), dtype=torch.float64, device="cuda:0")
        rr = torch.zeros(n, dtype=torch.float64, device="cuda:0")
        used = torch.zeros(n, dtype=torch.int32, device="cuda:0")
        mm.st_rom_surrogate_infer(n, dev_tensor(np.asarray(mu, dtype=np.float64)), dev_tensor(p.theta(mu)),
                                  1e30, uh, rr, used)
        mm.st_sync()
        outs.append(uh.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    # the loaded model's FOM march equals the original's (same operator)
    s1 = torch.zeros((1, 5, p.N), dtype=torch.float64, device="cuda:0")
    s2 = torch.zeros_like(s1)
    m.st_fom_march(p.theta(mu[:1]), p.dt[:5], None, dev_B(p), p.F[:5], s1)
    m2.st_fom_march(p.theta(mu[:1]), p.dt[:5], None, dev_B(p), p.F[:5], s2)
    m.st_sync()
    m2.st_sync()
    assert torch.equal(s1, s2)
    m.close()
    m2.close()


def test_resumed_build_equals_uninterrupted(c1, tmp_path):
    torch = __import__("torch")
    import paper_1910_01260_gb300 as st
    p, blocks = c1
    n_mu, Nt = len(blocks), p.Nt
    U = _snaps(blocks)
    # uninterrupted: one sample's snapshots per update
    ref = make_model(p, r_max=200)
    sig_ref, r_ref = ref.st_rom_build_basis(n_mu, Nt, U, p.ns, p.nt)
    # first half, saved; second half after loading
    a = make_model(p, r_max=200)
    a.st_pod_reset()
    a.st_pod_update(2 * Nt, U[:2], Nt)
    assert a.st_pod_get_dims()[1] == 2 * Nt
    path = tmp_path / "half.strom"
    a.st_model_save(str(path))
    assert st.st_model_file_info(str(path))["pod_rows"] == 2 * Nt
    b = st.Model.st_model_load(str(path), stream=torch.cuda.current_stream().cuda_stream)
    b.st_pod_update(2 * Nt, U[2:], Nt)
    b.st_pod_finish(n_mu, Nt, p.ns, p.nt)
    b.st_sync()
    sig_b, r_b = b.st_pod_get_state()
    assert r_b == r_ref and np.array_equal(sig_b, sig_ref)
    W1 = torch.zeros((r_ref, p.N), dtype=torch.float64, device="cuda:0")
    V1 = torch.zeros((r_ref, n_mu * Nt), dtype=torch.float64, device="cuda:0")
    W2, V2 = torch.zeros_like(W1), torch.zeros_like(V1)
    ref.st_pod_get_state(W1, V1)
    b.st_pod_get_state(W2, V2)
    assert torch.equal(W1, W2) and torch.equal(V1, V2)
    phi1 = torch.zeros((p.ns, p.N), dtype=torch.float64, device="cuda:0")
    T1 = torch.zeros((p.ns * p.nt, Nt), dtype=torch.float64, device="cuda:0")
    phi2, T2 = torch.zeros_like(phi1), torch.zeros_like(T1)
    ref.st_model_get_basis(phi1, T1)
    b.st_model_get_basis(phi2, T2)
    torch.cuda.synchronize()
    assert torch.equal(phi1, phi2) and torch.equal(T1, T2)
    # the same build fed group by group without saving also agrees
    c = make_model(p, r_max=200)
    for k in range(n_mu):
        c.st_pod_update(Nt, U[k:k + 1], Nt)
    c.st_pod_finish(n_mu, Nt, p.ns, p.nt)
    sig_c, r_c = c.st_pod_get_state()
    assert r_c == r_ref and np.array_equal(sig_c, sig_ref)
    for mm in (ref, a, b, c):
        mm.close()


def test_pod_finish_and_set_state_arguments(c1):
    import paper_1910_01260_gb300 as st
    p, blocks = c1
    m = make_model(p, r_max=200)
    m.st_pod_update(p.Nt, _snaps(blocks[:1]), p.Nt)
    with pytest.raises(st.StError) as e:   # 2 samples claimed, 1 consumed
        m.st_pod_finish(2, p.Nt, p.ns, 2)
    assert e.value.code == st.ST_ERR_ARG
    with pytest.raises(st.StError) as e:
        m.st_pod_update(p.Nt, _snaps(blocks[:1]), 0)
    assert e.value.code == st.ST_ERR_ARG
    with pytest.raises(st.StError) as e:   # increasing singular values
        m.st_pod_set_state(2, 0, dev_tensor(np.zeros((2, p.N))), np.array([1.0, 2.0]), None)
    assert e.value.code == st.ST_ERR_ARG
    m.close()
