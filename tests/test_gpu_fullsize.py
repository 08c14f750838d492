"""Parity at the benchmark's full sizes and launch configuration (2-D S4
transport, N = 49,152, Nt = 200, 16 training parameters, (40, 12) basis,
4096 online parameters with uneven sizes): sampled outputs the oracle can
compute one by one, and properties that hold at any size."""
import numpy as np
import pytest

from gpu_util import dev_B, dev_tensor, make_model, rel_max
from oracle import fom, strom
from workloads import c4_batch, problem_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c4():
    return problem_for("c4")


def test_fom_and_pod_full_size(c4):
    torch = __import__("torch")
    p = c4
    m = make_model(p, r_max=256)
    n = len(p.train_mu)
    snaps = torch.empty((n, p.Nt, p.N), dtype=torch.float64, device="cuda:0")
    status = torch.full((n,), -1, dtype=torch.int32, device="cuda:0")
    m.st_fom_march(p.theta(p.train_mu), p.dt, None, dev_B(p), p.F, snaps, None, status)
    torch.cuda.synchronize()
    assert int(status.abs().max()) == 0
    # sampled parameter: its first 60 steps by the oracle's sparse LU
    k = 5
    A = fom.affine_operator(p.rowptr, p.col, p.vals, p.theta(p.train_mu[k]))
    ref = fom.fom_march(A, p.dt[:60], p.B, p.F[:60], None)
    assert rel_max(snaps[k, :60].cpu().numpy().T, ref) < 1e-10
    sig, r = m.st_rom_build_basis(n, p.Nt, snaps, p.ns, p.nt)
    assert r == 256
    # leading singular values against the Gram matrix of the whole snapshot set
    U = snaps.reshape(n * p.Nt, p.N)
    lam = torch.linalg.eigvalsh(U @ U.T).flip(0).cpu().numpy()
    s_ref = np.sqrt(np.maximum(lam[:20], 0))
    assert np.abs(sig[:20] - s_ref).max() < 1e-9 * s_ref[0]
    phi = torch.zeros((p.ns, p.N), dtype=torch.float64, device="cuda:0")
    T = torch.zeros((p.ns * p.nt, p.Nt), dtype=torch.float64, device="cuda:0")
    m.st_model_get_basis(phi, T)
    Phi, Tm = phi.cpu().numpy().T, T.cpu().numpy().T
    # orthonormal to rounding of N-term FP64 sums (eps * sqrt(N) scale)
    assert np.abs(Phi.T @ Phi - np.eye(p.ns)).max() < 1e-11
    for i in range(p.ns):
        Ti = Tm[:, i::p.ns]
        assert np.abs(Ti.T @ Ti - np.eye(p.nt)).max() < 1e-12
    # Eckart-Young: the basis captures the snapshot energy up to the tail
    Ph = torch.tensor(Phi, device="cuda:0")
    resid = torch.linalg.norm(U.T - Ph @ (Ph.T @ U.T)) ** 2
    assert abs(resid.item() - (s_ref[p.ns:] ** 2).sum()) < 1e-6 * (s_ref ** 2).sum() + 1e-6 * resid.item()
    m.close()


def test_online_phase_full_size_sampled(c4):
    """Seeded orthonormal bases of the full size -> GPU assembly, solve of the
    whole 4096-parameter batch and reconstruction; 48 sampled parameters are
    recomputed by the oracle."""
    torch = __import__("torch")
    p = c4
    rng = np.random.default_rng(1)
    Phi = np.linalg.qr(rng.standard_normal((p.N, p.ns)))[0]
    T = np.zeros((p.Nt, p.ns * p.nt))
    for i in range(p.ns):
        T[:, i::p.ns] = np.linalg.qr(rng.standard_normal((p.Nt, p.nt)))[0]
    m = make_model(p)
    m.st_model_set_basis(p.ns, p.nt, p.Nt, dev_tensor(Phi.T.copy()), dev_tensor(T.T.copy()))
    m.st_rom_assemble(p.dt, dev_B(p), p.F, None)
    mu, sizes = c4_batch(4096, p)
    nf = p.ns * p.nt
    uhat = torch.zeros((4096, nf), dtype=torch.float64, device="cuda:0")
    res = torch.zeros(4096, dtype=torch.float64, device="cuda:0")
    status = torch.full((4096,), -1, dtype=torch.int32, device="cuda:0")
    m.st_rom_solve(4096, dev_tensor(p.theta(mu)), dev_tensor(sizes), uhat, res, status)
    y = torch.zeros((4096, p.Nt, 1), dtype=torch.float64, device="cuda:0")
    Cout = (np.repeat(p.w, p.n_cells) / p.n_cells)[None, :]
    m.st_rom_reconstruct(4096, uhat, dev_tensor(sizes), None, 1, dev_tensor(Cout), y)
    torch.cuda.synchronize()
    assert int((status != 0).sum()) == 0
    assert res.max().item() < 1e-11
    rm = strom.ReducedModel(p, Phi, T, p.ns, p.nt)
    Ahat, G, M, S, rhs = m.st_model_get_reduced(p.ns, p.nt)
    assert rel_max(Ahat, rm.Ahat_q) < 1e-12 and rel_max(G, rm.G) < 1e-12
    assert rel_max(rhs, rm.fhat) < 1e-12
    U = uhat.cpu().numpy()
    Y = y.cpu().numpy()
    for k in np.random.default_rng(2).choice(4096, 48, replace=False):
        a, b = sizes[k]
        want = rm.solve(p.theta(mu[k]), int(a), int(b))
        assert rel_max(U[k, :a * b], want) < 1e-10
        Uk = rm.reconstruct(want, int(a), int(b))
        assert rel_max(Y[k, :, 0], (Cout @ Uk)[0]) < 1e-9
    m.close()
