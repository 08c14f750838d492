"""End-to-end parity: FOM march -> POD -> assembly -> batched solve ->
reconstruction, all on the GPU through the C ABI, against the oracle doing
the same steps on the CPU (1-D slab workload, full size), plus the ROM error
against the FOM at unseen parameters.

Tolerance of the end-to-end fields: the GPU and oracle bases agree to
~1e-12 (singular vectors with relative gaps > 1e-2), the reduced operators
inherit that, and the reduced solve is well conditioned, so 1e-8 relative on
the reconstructed space-time field."""
import numpy as np
import pytest

from gpu_util import dev_B, dev_tensor, gpu_fom, make_model, oracle_fom, rel_max
from oracle import pod, strom
from workloads import problem_for

pytestmark = pytest.mark.gpu


def test_c1_end_to_end():
    torch = __import__("torch")
    p = problem_for("c1")
    m = make_model(p, r_max=200)
    B = dev_B(p)
    nmu = len(p.train_mu)
    snaps = torch.empty((nmu, p.Nt, p.N), dtype=torch.float64, device="cuda:0")
    m.st_fom_march(p.theta(p.train_mu), p.dt, None, B, p.F, snaps)
    sig, r = m.st_rom_build_basis(nmu, p.Nt, snaps, p.ns, p.nt)
    m.st_rom_assemble(p.dt, B, p.F, None)
    mus = p.test_mu
    n = len(mus)
    uhat = torch.zeros((n, p.ns * p.nt), dtype=torch.float64, device="cuda:0")
    res = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    m.st_rom_solve(n, dev_tensor(p.theta(mus)), None, uhat, res)
    U = torch.zeros((n, p.Nt, p.N), dtype=torch.float64, device="cuda:0")
    m.st_rom_reconstruct(n, uhat, None, U)
    m.st_sync()
    U = U.cpu().numpy()
    # oracle end to end
    blocks = oracle_fom(p, p.train_mu)
    ref = pod.pod_block_incremental(blocks, p.ns, p.nt, r_max=200)
    assert np.abs(sig[:40] - ref["sigma"][:40]).max() < 1e-11 * ref["sigma"][0]
    rm = strom.ReducedModel(p, ref["Phi_s"], ref["T"], p.ns, p.nt)
    fom_test, _, _ = gpu_fom(m, p, mus)
    for k in range(n):
        want = rm.reconstruct(rm.solve(p.theta(mus[k])))
        assert rel_max(U[k].T, want) < 1e-8
        # ROM accuracy against the FOM (measured outcome, loose bound)
        assert strom.rel_error(fom_test[k], U[k].T) < 1e-2
    assert res.max().item() < 1e-12
    m.close()


def test_profile_and_pod_stats():
    """Per-kernel event timing covers the launches of every stage, GEMM and
    Jacobi flops are counted, and the POD diagnostics match the update count."""
    torch = __import__("torch")
    p = problem_for("c1")
    m = make_model(p, r_max=200)
    B = dev_B(p)
    nmu = len(p.train_mu)
    snaps = torch.empty((nmu, p.Nt, p.N), dtype=torch.float64, device="cuda:0")
    m.st_profile_enable(True)
    m.st_fom_march(p.theta(p.train_mu), p.dt, None, B, p.F, snaps)
    m.st_rom_build_basis(nmu, p.Nt, snaps, p.ns, p.nt)
    m.st_rom_assemble(p.dt, B, p.F, None)
    uhat = torch.zeros((3, p.ns * p.nt), dtype=torch.float64, device="cuda:0")
    m.st_rom_solve(3, dev_tensor(p.theta(p.test_mu[:3])), None, uhat)
    prof = m.st_profile_read()
    for name in ("fom_march_kernel", "jacobi_kernel", "solve_kernel<double>", "gs2_kernel"):
        assert name in prof and prof[name][0] > 0.0 and prof[name][1] >= 1, name
    gemm = [v for k, v in prof.items() if k.startswith("dgemm_kernel[")]
    assert gemm and all(v[0] > 0.0 and v[2] > 0 for v in gemm)
    assert prof["jacobi_kernel"][2] > 0
    times = [v[0] for v in prof.values()]
    assert times == sorted(times, reverse=True)
    sweeps, reorth = m.st_pod_get_stats()
    assert len(sweeps) == nmu and all(1 <= s <= 40 for s in sweeps) and reorth >= 0
    assert prof["jacobi_kernel"][1] == nmu
    m.st_profile_enable(False)
    m.st_rom_solve(3, dev_tensor(p.theta(p.test_mu[:3])), None, uhat)
    assert m.st_profile_read() == {}
    m.close()
