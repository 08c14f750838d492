"""Pins of the oracle's POD (Sec. 4.1) and incremental SVD (Sec. 4.2): block
updates and the rank-one streaming update of Algorithm 2."""
import numpy as np
import pytest

from oracle import fom, pod
from workloads import make_problem, problem_for


@pytest.fixture(scope="module")
def c1_blocks():
    p = problem_for("c1")
    blocks = [fom.fom_march(fom.affine_operator(p.rowptr, p.col, p.vals, p.theta(mu)),
                            p.dt, p.B, p.F, p.u0) for mu in p.train_mu]
    return p, blocks


def test_exact_pod_identities(c1_blocks):
    p, blocks = c1_blocks
    U = pod.snapshot_matrix(blocks)
    r = pod.pod_exact(blocks, p.ns, p.nt)
    W, s, V = r["W"], r["sigma"], r["V"]
    assert np.abs(W.T @ W - np.eye(W.shape[1])).max() < 1e-13
    assert np.abs(V.T @ V - np.eye(V.shape[1])).max() < 1e-13
    # Eq. SVDsummation and sum sigma^2 = ||U||_F^2
    assert np.abs(W @ np.diag(s) @ V.T - U).max() < 1e-12 * s[0]
    assert abs((s ** 2).sum() - np.linalg.norm(U) ** 2) < 1e-12 * (s ** 2).sum()
    # Eckart-Young optimality of Eq. POD: the residual energy is the tail
    for ns in (1, 4, 8, 20):
        Ph = W[:, :ns]
        res = np.linalg.norm(U - Ph @ (Ph.T @ U)) ** 2
        assert abs(res - (s[ns:] ** 2).sum()) < 1e-10 * (s ** 2).sum()
    # no other orthonormal basis of the same size does better
    rng = np.random.default_rng(0)
    X, _ = np.linalg.qr(W[:, :8] + 1e-3 * rng.standard_normal(W[:, :8].shape))
    assert np.linalg.norm(U - X @ (X.T @ U)) ** 2 > (s[8:] ** 2).sum()


def test_temporal_snapshot_indexing(c1_blocks):
    # v_i^k is the k-th length-Nt segment of v_i, so by Eq. SVDsummation
    # U_k = sum_i sigma_i w_i (v_i^k)^T, i.e. column k of Upsilon_i.
    p, blocks = c1_blocks
    r = pod.pod_exact(blocks, p.ns, p.nt)
    W, s, V = r["W"], r["sigma"], r["V"]
    n_mu, Nt = len(blocks), p.Nt
    ups = [V[:, i].reshape(n_mu, Nt).T for i in range(len(s))]
    for k in range(n_mu):
        Uk = sum(s[i] * np.outer(W[:, i], ups[i][:, k]) for i in range(len(s)))
        assert np.abs(Uk - blocks[k]).max() < 1e-11 * s[0]
    T = r["T"]
    for i in range(p.ns):
        Ti = T[:, [i + p.ns * j for j in range(p.nt)]]
        assert np.abs(Ti.T @ Ti - np.eye(p.nt)).max() < 1e-13
        # Phi_t^i spans the dominant left singular space of Upsilon_i
        lam, sv, _ = np.linalg.svd(ups[i], full_matrices=False)
        assert np.abs(Ti @ Ti.T - lam[:, :p.nt] @ lam[:, :p.nt].T).max() < 1e-10
        assert np.allclose(r["temporal_sigma"][i], sv[:r["temporal_sigma"].shape[1]])


def test_incremental_equals_exact_when_untruncated(c1_blocks):
    p, blocks = c1_blocks
    ex = pod.pod_exact(blocks, p.ns, p.nt)
    inc = pod.pod_block_incremental(blocks, p.ns, p.nt, r_max=10 ** 6, eps_svd=1e-14,
                                    eps_sv=1e-15)
    k = 40
    s0 = ex["sigma"][0]
    assert np.abs(inc["sigma"][:k] - ex["sigma"][:k]).max() < 1e-12 * s0
    # leading spatial modes (distinct singular values) agree up to sign
    assert np.abs(pod.canonical_signs(inc["Phi_s"]) - pod.canonical_signs(ex["Phi_s"])).max() < 1e-9
    # temporal bases: compare projectors, which do not depend on signs
    for i in range(p.ns):
        cols = [i + p.ns * j for j in range(p.nt)]
        Pe = ex["T"][:, cols] @ ex["T"][:, cols].T
        Pi = inc["T"][:, cols] @ inc["T"][:, cols].T
        assert np.abs(Pe - Pi).max() < 1e-8
    W = inc["W"]
    assert np.abs(W.T @ W - np.eye(W.shape[1])).max() < 1e-12


def test_incremental_truncated_keeps_leading_modes(c1_blocks):
    p, blocks = c1_blocks
    ex = pod.pod_exact(blocks, p.ns, p.nt)
    inc = pod.pod_block_incremental(blocks, p.ns, p.nt, r_max=60)
    assert inc["W"].shape[1] == 60
    s0 = ex["sigma"][0]
    assert np.abs(inc["sigma"][:8] - ex["sigma"][:8]).max() < 1e-9 * s0
    U = pod.snapshot_matrix(blocks)
    approx = inc["W"] @ np.diag(inc["sigma"]) @ inc["V"].T
    # truncation only removes small singular directions
    assert np.linalg.norm(U - approx) < 1e-3 * np.linalg.norm(U)


def test_incremental_dependent_and_zero_columns():
    rng = np.random.default_rng(7)
    base = rng.standard_normal((40, 3))
    b1 = base @ rng.standard_normal((3, 6))          # rank 3 block
    b2 = np.zeros((40, 6))                           # all-zero block
    b3 = np.concatenate([b1[:, :2], rng.standard_normal((40, 4))], axis=1)
    blocks = [b1, b2, b3]
    ex = pod.pod_exact(blocks, 3, 2)
    inc = pod.pod_block_incremental(blocks, 3, 2, r_max=100)
    rank = np.linalg.matrix_rank(pod.snapshot_matrix(blocks))
    assert inc["W"].shape[1] == rank == 7
    assert np.abs(inc["sigma"] - ex["sigma"][:rank]).max() < 1e-12 * ex["sigma"][0]
    approx = inc["W"] @ np.diag(inc["sigma"]) @ inc["V"].T
    assert np.abs(approx - pod.snapshot_matrix(blocks)).max() < 1e-12 * ex["sigma"][0]


def test_canonical_signs():
    X = np.array([[1.0, -3.0], [-2.0, 1.0], [0.5, 3.0]])
    C = pod.canonical_signs(X)
    assert np.allclose(C[:, 0], -X[:, 0]) and np.allclose(C[:, 1], -X[:, 1])
    assert np.allclose(pod.canonical_signs(-X), C)


# ---- the rank-one streaming update of Algorithm 2 (one snapshot per update) ----

def test_rank_one_stream_equals_exact_when_untruncated(c1_blocks):
    p, blocks = c1_blocks
    ex = pod.pod_exact(blocks, p.ns, p.nt)
    inc = pod.pod_block_incremental(blocks, p.ns, p.nt, r_max=10 ** 6, eps_svd=1e-14,
                                    eps_sv=1e-15, cols_per_update=1)
    k = 40
    s0 = ex["sigma"][0]
    assert np.abs(inc["sigma"][:k] - ex["sigma"][:k]).max() < 1e-12 * s0
    assert np.abs(pod.canonical_signs(inc["Phi_s"]) - pod.canonical_signs(ex["Phi_s"])).max() < 1e-9
    for i in range(p.ns):
        cols = [i + p.ns * j for j in range(p.nt)]
        Pe = ex["T"][:, cols] @ ex["T"][:, cols].T
        Pi = inc["T"][:, cols] @ inc["T"][:, cols].T
        assert np.abs(Pe - Pi).max() < 1e-8
    # U = W Sigma V^T with V's rows in snapshot-column order (Eq. SVDsummation)
    U = pod.snapshot_matrix(blocks)
    assert np.abs(inc["W"] @ np.diag(inc["sigma"]) @ inc["V"].T - U).max() < 1e-11 * s0


def test_rank_one_stream_on_a_hand_sized_case():
    # three snapshots in R^3 with a dependent third one: after the rank-one
    # updates the SVD is that of the 3 x 3 matrix, of rank 2
    U = np.array([[3.0, 0.0, 6.0], [4.0, 0.0, 8.0], [0.0, 2.0, 0.0]])
    inc = pod.pod_block_incremental([U], 1, 1, r_max=10, cols_per_update=1)
    # columns u1 = (3,4,0), u2 = (0,0,2), u3 = 2 u1: U^T U = diag-free Gram of
    # rank 2 with singular values sqrt(25 + 100) = sqrt(125) and 2
    assert inc["W"].shape[1] == 2
    assert np.allclose(inc["sigma"], [np.sqrt(125.0), 2.0], rtol=0, atol=1e-14)
    assert np.abs(inc["W"] @ np.diag(inc["sigma"]) @ inc["V"].T - U).max() < 1e-14


def test_rank_one_stream_truncated_keeps_leading_modes(c1_blocks):
    p, blocks = c1_blocks
    ex = pod.pod_exact(blocks, p.ns, p.nt)
    inc = pod.pod_block_incremental(blocks, p.ns, p.nt, r_max=60, cols_per_update=1)
    assert inc["W"].shape[1] == 60
    s0 = ex["sigma"][0]
    assert np.abs(inc["sigma"][:8] - ex["sigma"][:8]).max() < 1e-9 * s0
    U = pod.snapshot_matrix(blocks)
    approx = inc["W"] @ np.diag(inc["sigma"]) @ inc["V"].T
    assert np.linalg.norm(U - approx) < 1e-3 * np.linalg.norm(U)


# ---- the orthogonality check and re-orthogonalisation that end Algorithm 2 ----

def _upper_perturbed_basis(n, r, delta, seed=3):
    """W = Q0 R0 with Q0 orthonormal and R0 = I + delta * (strictly upper
    triangular, entries in [1, 2)): by uniqueness of the QR factorisation with a
    positive R diagonal, the re-orthogonalisation of W must return Q0 exactly
    (to rounding), and w_1^T w_r = R0[0, r-1]."""
    rng = np.random.default_rng(seed)
    Q0 = np.linalg.qr(rng.standard_normal((n, r)))[0]
    R0 = np.eye(r) + delta * np.triu(1.0 + rng.random((r, r)), 1)
    return Q0, R0, Q0 @ R0


@pytest.mark.parametrize("delta", [1e-6, -1e-6, 1e-9])
def test_orthogonality_check_returns_the_positive_qr_factor(delta):
    n, r = 300, 7
    Q0, R0, W = _upper_perturbed_basis(n, r, delta)
    assert abs(W[:, 0] @ W[:, -1] - R0[0, -1]) < 1e-15
    Wq, fired = pod.orthogonality_check(W, eps_svd=1e-12)
    # the test reads |w_1^T w_r|: a negative inner product fires as well
    assert fired
    # Q0 itself: a column with the wrong sign (R with a negative diagonal), a
    # factor of W^T instead of W, or a skipped step all miss this by >= delta
    assert np.abs(Wq - Q0).max() < 1e-14
    assert np.abs(Wq.T @ Wq - np.eye(r)).max() < 1e-15 * n
    # W = Wq R0: each column keeps its span with the earlier ones and its sign
    assert np.abs(Wq.T @ W - R0).max() < 1e-14


def test_orthogonality_check_threshold():
    n, r = 300, 5
    thr = min(1e-12, pod.EPS * n)               # 3.3e-14 at n = 300
    Q0, R0, W = _upper_perturbed_basis(n, r, 0.0)
    W[:, -1] += 0.5 * thr * W[:, 0]             # |w_1^T w_r| = thr / 2: no action
    Wq, fired = pod.orthogonality_check(W, eps_svd=1e-12)
    assert not fired and Wq is W
    W[:, -1] += 2.0 * thr * W[:, 0]             # 2.5 thr: fires
    assert pod.orthogonality_check(W, eps_svd=1e-12)[1]
    # eps_svd below eps * N sets the threshold
    W2 = Q0.copy()
    W2[:, -1] += 1e-15 * W2[:, 0]
    assert not pod.orthogonality_check(W2, eps_svd=1e-3)[1]
    assert pod.orthogonality_check(W2, eps_svd=1e-16)[1]
    # a single column is never tested
    assert not pod.orthogonality_check(W[:, :1] * 3.0, eps_svd=0.0)[1]


def test_incremental_update_reorthogonalises_a_drifted_basis(c1_blocks):
    """A basis that has lost orthogonality (W = W0 (I + delta U), U strictly
    upper triangular) enters an update: the update must end orthonormal, keep
    each column's orientation, and still factorise the data up to O(delta)."""
    p, blocks = c1_blocks
    W0, s0, V0 = pod.incremental_update(None, None, None, blocks[0], 200, 1e-12, 1e-14)
    r = W0.shape[1]
    rng = np.random.default_rng(11)
    delta = 1e-7
    Wd = W0 @ (np.eye(r) + delta * np.triu(rng.random((r, r)), 1))
    W_ref, s_ref, V_ref = pod.incremental_update(W0, s0, V0, blocks[1], 200, 1e-12, 1e-14)
    W_d, s_d, V_d = pod.incremental_update(Wd, s0, V0, blocks[1], 200, 1e-12, 1e-14)
    # without step 6 the drift of the input would survive at ~delta
    assert np.abs(W_d.T @ W_d - np.eye(W_d.shape[1])).max() < 1e-13
    k = min(10, W_d.shape[1])
    # the leading directions keep their orientation (no sign flips)
    assert np.all(np.einsum("ij,ij->j", W_d[:, :k], W_ref[:, :k]) > 0.99)
    U = pod.snapshot_matrix(blocks[:2])
    err = np.abs(W_d @ np.diag(s_d) @ V_d.T - U).max() / s_d[0]
    assert err < 100 * delta
    # the exact-arithmetic path does not fire on these snapshots
    assert np.abs(W_ref.T @ W_ref - np.eye(W_ref.shape[1])).max() < 1e-13
