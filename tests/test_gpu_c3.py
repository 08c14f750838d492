"""Config c3 at its full size (2-D S6 transport on 256 x 256 cells, N =
1,572,864, 40.9 M stored entries): the GPU march against the oracle's
textbook BiCGSTAB (tolerance 1e-14) on the first steps of a training
parameter.  A direct sparse factorisation of this operator is beyond the
host, so the oracle's iterative solver is the reference here; its own pins
(against the sparse LU and the dense solve) are in tests/test_oracle_fom.py."""
import numpy as np
import pytest

from gpu_util import gpu_fom, make_model, rel_max
from oracle import fom
from workloads import problem_for

pytestmark = pytest.mark.gpu


def test_c3_first_steps_against_the_oracle():
    p = problem_for("c3")
    K = 3
    mus = p.train_mu[[0, 31]]
    m = make_model(p)
    got, status, it = gpu_fom(m, p, mus, Nt=K, with_iters=True)
    assert (status == 0).all()
    for k in (0, 1):
        A = fom.affine_operator(p.rowptr, p.col, p.vals, p.theta(mus[k]))
        ref = fom.fom_march(A, p.dt[:K], p.B, p.F[:K], None, solver="bicgstab", tol=1e-14, maxit=500)
        assert rel_max(got[k], ref) < 1e-10
    m.close()
