"""The stability constant of Theorem 3 on the GPU: the power-iteration
estimate of ||(A^st)^-1||_2 (forward march + transposed march backward in
time) against the dense singular values of the assembled space-time matrix
(small cases), and the complete a posteriori certificate -- library residual
norms times the library's constant -- bounding the true ROM error."""
import numpy as np
import pytest

from gpu_util import dev_B, dev_tensor, make_model, oracle_fom
from oracle import fom, pod, strom
from workloads import make_problem

pytestmark = pytest.mark.gpu


def _dense_inverse_norm(p, theta):
    A = fom.affine_operator(p.rowptr, p.col, p.vals, theta)
    Ast, _ = fom.st_fom_system(A, p.dt, p.B, p.F, None)
    return 1.0 / np.linalg.svd(Ast.toarray(), compute_uv=False).min()


@pytest.mark.parametrize("case", ["1d", "2d"])
def test_inverse_norm_matches_the_dense_singular_value(case):
    if case == "1d":
        p = make_problem(dim=1, M=8, quad="gl4", Nt=6, g="sin", ns=3, nt=2)
    else:
        p = make_problem(dim=2, M=4, quad="s4", Nt=8, source="gaussian", g="ramp", ns=3, nt=2)
    th = p.theta(np.concatenate([p.train_mu, p.test_mu])[:5])
    m = make_model(p)
    est, it = m.st_fom_st_inverse_norm(th, p.dt, max_iter=2000, tol=1e-12)
    for k in range(len(th)):
        want = _dense_inverse_norm(p, th[k])
        # a lower estimate converging from below
        assert est[k] <= want * (1 + 1e-12)
        assert abs(est[k] - want) < 1e-6 * want, (k, est[k], want, it)
    m.close()


def test_theorem3_certificate_from_library_quantities():
    import torch
    p = make_problem(dim=1, M=8, quad="gl4", Nt=6, g="sin", ns=3, nt=2)
    blocks = oracle_fom(p, p.train_mu)
    ref = pod.pod_exact(blocks, p.ns, p.nt)
    m = make_model(p)
    m.st_model_set_basis(p.ns, p.nt, p.Nt, dev_tensor(ref["Phi_s"].T.copy()), dev_tensor(ref["T"].T.copy()))
    m.st_rom_assemble(p.dt, dev_B(p), p.F, None)
    th = p.theta(p.test_mu)
    n, nf = len(th), p.ns * p.nt
    uh = torch.zeros((n, nf), dtype=torch.float64, device="cuda:0")
    m.st_rom_solve(n, dev_tensor(th), None, uh)
    U = torch.zeros((n, p.Nt, p.N), dtype=torch.float64, device="cuda:0")
    m.st_rom_reconstruct(n, uh, None, U)
    rn = torch.zeros((n, p.Nt), dtype=torch.float64, device="cuda:0")
    m.st_rom_residual_norms(th, p.dt, None, dev_B(p), p.F, U, rn)
    m.st_sync()
    const, _ = m.st_fom_st_inverse_norm(th, p.dt, max_iter=2000, tol=1e-12)
    Ug = U.cpu().numpy()
    R = rn.cpu().numpy()
    for k in range(n):
        A = fom.affine_operator(p.rowptr, p.col, p.vals, th[k])
        Uf = fom.fom_march(A, p.dt, p.B, p.F, None, solver="dense")
        err = strom.st_inf_norm(Uf - Ug[k].T)
        bound = np.sqrt(p.Nt) * const[k] * R[k].max()
        assert err > 1e-8 * np.abs(Uf).max()
        assert err <= bound * (1 + 1e-6)
    m.close()


def test_inverse_norm_arguments():
    import paper_1910_01260_gb300 as st
    p = make_problem(dim=1, M=8, quad="gl4", Nt=6, ns=3, nt=2)
    m = make_model(p)
    with pytest.raises(st.StError) as e:
        m.st_fom_st_inverse_norm(p.theta(p.test_mu[:1]), -p.dt)
    assert e.value.code == st.ST_ERR_ARG
    with pytest.raises(st.StError) as e:
        m.st_fom_st_inverse_norm(p.theta(p.test_mu[:1]), p.dt, max_iter=1, tol=0.0)
    assert e.value.code == st.ST_ERR_NOT_CONVERGED
    m.close()
