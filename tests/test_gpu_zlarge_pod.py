"""The Gram-Schmidt kernel's variant for long columns: at c3's N = 1,572,864
a CTA owns 10,348 rows, and three columns of them (248 KB) exceed the
shared memory of an SM, so the kernel keeps the columns of E in global
memory and only its first two directions in shared memory.  A first
incremental-SVD update of synthetic columns with a decaying spectrum is
checked against the oracle's update of the same columns (Sec. 4.2): singular
values, orthonormality of W, and the factorisation itself.  Singular vectors
are not compared: the spectrum's relative gaps (about 0.44 sigma_i) bound
them only loosely through W Sigma V^T."""
import numpy as np
import pytest

from gpu_util import dev_tensor, make_model
from oracle import pod
from workloads import problem_for

pytestmark = pytest.mark.gpu


def test_first_update_with_columns_longer_than_shared_memory():
    torch = __import__("torch")
    p = problem_for("c3")  # its operator only sizes the model
    N, n = p.N, 24
    rng = np.random.default_rng(21)
    s = 10.0 ** (-0.25 * np.arange(n))
    Y = np.linalg.qr(rng.standard_normal((n, n)))[0]
    U = (rng.standard_normal((N, n)) * s) @ Y.T
    W_o, s_o, V_o = pod.incremental_update(None, None, None, U, 64, 1e-12, 1e-14)
    assert len(s_o) == n
    m = make_model(p, r_max=64)
    m.st_pod_update(n, dev_tensor(U.T.copy()), n)
    r, rows = m.st_pod_get_dims()
    assert (r, rows) == (n, n)
    W = torch.zeros((r, N), dtype=torch.float64, device="cuda:0")
    V = torch.zeros((r, n), dtype=torch.float64, device="cuda:0")
    sig, r2 = m.st_pod_get_state(W, V)
    assert r2 == r
    Wg, Vg = W.cpu().numpy().T, V.cpu().numpy().T
    assert np.abs(sig - s_o).max() < 1e-11 * s_o[0]
    assert np.abs(Wg.T @ Wg - np.eye(r)).max() < 1e-12
    assert np.abs(Vg.T @ Vg - np.eye(r)).max() < 1e-12
    assert np.abs(Wg @ np.diag(sig) @ Vg.T - U).max() < 1e-11 * s_o[0]
    m.close()
