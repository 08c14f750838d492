"""Parity at the benchmark's full sizes and launch configuration (2-D S4
transport, N = 49,152, Nt = 200, 16 training parameters, (40, 12) basis,
4096 online parameters with uneven sizes): sampled outputs the oracle can
compute one by one, and properties that hold at any size."""
import numpy as np
import pytest

from gpu_util import dev_B, dev_tensor, make_model, oracle_fom_train_parallel, rel_max
from oracle import fom, pod, strom
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


# the benchmark's incremental-SVD settings: updates of 8 samples (1,600
# snapshot columns), the paper's first example's eps_svd, r_max = 256
BENCH_POD = dict(pod_block=8, eps_svd=2e-8, r_max=256)


def test_pod_at_benchmark_settings(c4):
    """The basis the benchmark builds, compared with the oracle's incremental
    SVD of the same (oracle) snapshots at the same settings.  Singular values,
    the well-separated leading spatial modes, and the projections of the
    snapshots on the spatial and per-mode temporal bases are compared, then
    the ROM built on each basis: several spatial modes come in near-degenerate
    pairs and the temporal bases' last vectors sit at the noise level, so
    individual vectors there are not determined to rounding (the tolerance of
    a projection grows like rounding / gap)."""
    torch = __import__("torch")
    p = c4
    blocks = oracle_fom_train_parallel("c4")
    n, Nt = len(blocks), p.Nt
    ref = pod.pod_block_incremental(blocks, p.ns, p.nt, r_max=256, eps_svd=2e-8,
                                    cols_per_update=BENCH_POD["pod_block"] * Nt)
    m = make_model(p, **BENCH_POD)
    snaps = dev_tensor(np.stack([b.T for b in blocks]))
    sig, r = m.st_rom_build_basis(n, Nt, snaps, p.ns, p.nt)
    s_o = ref["sigma"]
    assert abs(r - len(s_o)) <= 2
    assert np.abs(sig[:40] - s_o[:40]).max() < 1e-11 * s_o[0]
    phi = torch.zeros((p.ns, p.N), dtype=torch.float64, device="cuda:0")
    T = torch.zeros((p.ns * p.nt, Nt), dtype=torch.float64, device="cuda:0")
    m.st_model_get_basis(phi, T)
    V = torch.zeros((r, n * Nt), dtype=torch.float64, device="cuda:0")
    m.st_pod_get_state(None, V)
    torch.cuda.synchronize()
    Phi, Tm, Vg = phi.cpu().numpy().T, T.cpu().numpy().T, V.cpu().numpy().T
    # gap of each spatial mode to its neighbours, relative to sigma_1
    gap = np.minimum(np.r_[np.inf, -np.diff(s_o)], np.r_[-np.diff(s_o), np.inf])[:p.ns] / s_o[0]
    lead = [i for i in range(p.ns) if gap[i] > 5e-3]
    assert len(lead) >= 4
    assert np.abs(pod.canonical_signs(Phi[:, lead]) - pod.canonical_signs(ref["Phi_s"][:, lead])).max() < 1e-9
    U = np.concatenate(blocks, axis=1)
    Ph, Po = Phi, ref["Phi_s"]
    d = np.linalg.norm(Ph @ (Ph.T @ U) - Po @ (Po.T @ U)) / np.linalg.norm(U)
    assert d < 1e-10
    # per-mode temporal bases: projection of the oracle's temporal snapshots
    for i in range(p.ns):
        ups = ref["V"][:, i].reshape(n, Nt).T
        cols = [i + p.ns * j for j in range(p.nt)]
        Tg, To = Tm[:, cols], ref["T"][:, cols]
        e = np.linalg.norm(Tg @ (Tg.T @ ups) - To @ (To.T @ ups)) / np.linalg.norm(ups)
        assert e < 1e-8 + 1e-12 / gap[i], (i, e)
    # the ROM on each basis: GPU assembly + solve + reconstruction against the
    # oracle's reduced model on its own basis, at (40, 12) and (20, 8)
    m.st_rom_assemble(p.dt, dev_B(p), p.F, None)
    rm = strom.ReducedModel(p, ref["Phi_s"], ref["T"], p.ns, p.nt)
    mu, _ = c4_batch(4, p)
    sizes = np.array([[40, 12], [20, 8], [40, 12], [20, 8]], dtype=np.int32)
    uh = torch.zeros((4, p.ns * p.nt), dtype=torch.float64, device="cuda:0")
    m.st_rom_solve(4, dev_tensor(p.theta(mu)), dev_tensor(sizes), uh)
    u = torch.zeros((4, Nt, p.N), dtype=torch.float64, device="cuda:0")
    m.st_rom_reconstruct(4, uh, dev_tensor(sizes), u)
    m.st_sync()
    for k in range(4):
        a, b = (int(x) for x in sizes[k])
        want = rm.reconstruct(rm.solve(p.theta(mu[k]), a, b), a, b)
        got = u[k].cpu().numpy().T
        assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-8
    m.close()


# FP64 LU; FP32 LU + 2 FP64 refinements (the benchmark's mode); + 3
@pytest.mark.parametrize("precision,refine", [(0, 1), (2, 2), (2, 3)])
def test_online_phase_full_size_sampled(c4, precision, refine):
    """Seeded orthonormal bases of the full size -> GPU assembly, solve of the
    whole 4096-parameter batch and reconstruction; 48 sampled parameters are
    recomputed by the oracle.  Run in the FP64 mode and in the benchmark's
    mode (FP32 LU factors, two FP64 residual refinements; also three), whose
    result must meet the FP64 tolerance at every size up to n = 480."""
    torch = __import__("torch")
    p = c4
    rng = np.random.default_rng(1)
    Phi = np.linalg.qr(rng.standard_normal((p.N, p.ns)))[0]
    T = np.zeros((p.Nt, p.ns * p.nt))
    for i in range(p.ns):
        T[:, i::p.ns] = np.linalg.qr(rng.standard_normal((p.Nt, p.nt)))[0]
    m = make_model(p, precision=precision, refine_steps=refine)
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
    # every sampled size class, with the largest (n = 480) included
    pick = list(np.random.default_rng(2).choice(4096, 48, replace=False))
    pick += [int(np.where((sizes[:, 0] == 40) & (sizes[:, 1] == 12))[0][j]) for j in range(4)]
    for k in pick:
        a, b = sizes[k]
        want = rm.solve(p.theta(mu[k]), int(a), int(b))
        assert rel_max(U[k, :a * b], want) < 1e-10
        Uk = rm.reconstruct(want, int(a), int(b))
        assert rel_max(Y[k, :, 0], (Cout @ Uk)[0]) < 1e-9
    m.close()
