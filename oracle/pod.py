"""Oracle: basis generation (Sec. 4).

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``pod_exact`` -- method of snapshots (Sec. 4.1): snapshot matrix
  U = [U_1 ... U_nmu] (Eq. snapshotmat), thin SVD U = W Sigma V^T (Eq. SVD,
  LAPACK via numpy), spatial basis Phi_s = W(:, 1:ns).
* ``temporal_bases`` -- per spatial mode i, the temporal snapshot matrix
  Upsilon_i = [v_i^1 ... v_i^nmu] with v_i^k = V((k-1) Nt + 1 : k Nt, i)
  (Eq. temporalSVD and the text before it), its SVD, and
  Phi_t^i = Lambda_i(:, 1:nt).  Stored as T (Nt x ns*nt) with column
  i + ns*j holding phi_t^{i,j} (index order of Eq. spacetimebasis).
* ``pod_block_incremental`` -- the incremental SVD of Sec. 4.2 (Eqs.
  factorization1 ... rankOneUpdateSVD2, Algorithms 1-2), taking one
  parameter's Nt snapshots per update (or any fixed number of consecutive
  snapshot columns; one column per update is Algorithm 2's rank-one update):
    1. project the block on W: L1 = W^T U_p, E1 = U_p - W L1;
    2. within the block, column by column, project each column of E1 on the
       new directions found so far (two passes), and keep its normalised
       remainder as a new direction unless its norm is below the dependence
       threshold (the "p < eps_SVD" test of Algorithm 2, read relative to the
       block's largest column norm); this gives E1 = J1 P1;
    2b. second block pass, the finite-precision safeguard of Sec. 4.2 taken
       as block Gram-Schmidt twice: a remainder normalised from a small norm
       amplifies its rounding along W, so J1 is projected on W again,
       L2 = W^T J1, and J1 - W L2 = J P2 is re-orthogonalised; then
       U_p = W L + J P with L = L1 + L2 P1 and P = P2 P1;
    3. SVD of the bordered middle matrix Q = [[diag(sigma), L], [0, P]]
       (Eq. middleMat, with a block border instead of one column);
    4. W <- [W J] Ubar, sigma <- diag(Sigma_bar), V <- blkdiag(V, I) Vbar
       (Eqs. rankOneUpdateSVD1-2);
    5. drop singular values below eps_SV * sigma_max and keep at most r_max;
    6. the orthogonality check of Algorithm 2 (|w_1^T w_end| > min(eps_SVD,
       eps * N)) followed by a QR re-orthogonalisation; the QR is taken with a
       positive diagonal in R so that no column of W changes sign (a sign flip
       of w_i without v_i would break W Sigma V^T).
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import numpy as np

EPS = 2.0 ** -53


def snapshot_matrix(blocks: Sequence[np.ndarray]) -> np.ndarray:
    """U = [U_1 ... U_nmu] (Eq. snapshotmat)."""
    return np.concatenate(list(blocks), axis=1)


def temporal_bases(V: np.ndarray, n_mu: int, Nt: int, ns: int, nt: int
                   ) -> Tuple[np.ndarray, np.ndarray]:
    """T (Nt x ns*nt) and the temporal singular values (ns x min(Nt, nmu)).

    Upsilon_i[:, k] = V[k*Nt:(k+1)*Nt, i] (unscaled right singular vector,
    Sec. 4.1), Phi_t^i = left singular vectors (:, :nt)."""
    T = np.zeros((Nt, ns * nt), dtype=np.float64)
    svals = np.zeros((ns, min(Nt, n_mu)), dtype=np.float64)
    for i in range(ns):
        ups = V[:, i].reshape(n_mu, Nt).T
        lam, s, _ = np.linalg.svd(ups, full_matrices=False)
        svals[i, :s.shape[0]] = s
        for j in range(nt):
            T[:, i + ns * j] = lam[:, j]
    return T, svals


def pod_exact(blocks: Sequence[np.ndarray], ns: int, nt: int) -> dict:
    """Exact POD of Sec. 4.1 (thin SVD of the whole snapshot matrix)."""
    U = snapshot_matrix(blocks)
    n_mu = len(blocks)
    Nt = blocks[0].shape[1]
    W, s, Vt = np.linalg.svd(U, full_matrices=False)
    V = Vt.T
    T, tsv = temporal_bases(V, n_mu, Nt, ns, nt)
    return dict(W=W, sigma=s, V=V, Phi_s=W[:, :ns].copy(), T=T, temporal_sigma=tsv)


def _colwise_gs2(E: np.ndarray, tau: float) -> Tuple[np.ndarray, np.ndarray]:
    """Column-by-column Gram-Schmidt with a second pass inside one block.
    Returns J (N x k, orthonormal) and P (k x m) with E = J P up to rounding;
    columns whose remainder norm is <= tau add no direction."""
    n, m = E.shape
    J = np.zeros((n, m), dtype=np.float64)
    P = np.zeros((m, m), dtype=np.float64)
    k = 0
    for j in range(m):
        e = E[:, j].copy()
        h = J[:, :k].T @ e
        e -= J[:, :k] @ h
        h2 = J[:, :k].T @ e
        e -= J[:, :k] @ h2
        h += h2
        nu = np.linalg.norm(e)
        P[:k, j] = h
        if nu > tau:
            J[:, k] = e / nu
            P[k, j] = nu
            k += 1
    return J[:, :k].copy(), P[:k, :].copy()


def incremental_update(W: Optional[np.ndarray], sigma: Optional[np.ndarray],
                       V: Optional[np.ndarray], Up: np.ndarray, r_max: int,
                       eps_svd: float, eps_sv: float):
    """One block update of the incremental SVD (steps 1-6 of the module
    docstring).  W, sigma, V are None before the first block."""
    n, m = Up.shape
    tau = eps_svd * float(np.max(np.linalg.norm(Up, axis=0))) if m else 0.0
    r = 0 if W is None else W.shape[1]
    if r > 0:
        # first block pass: project on W, orthogonalise the remainder
        L1 = W.T @ Up
        E1 = Up - W @ L1
        J1, P1 = _colwise_gs2(E1, tau)
        # second block pass: directions of E1 that were normalised from a
        # small remainder carry amplified rounding along W; project J1 on W
        # again and re-orthogonalise (U_p = W (L1 + L2 P1) + J (P2 P1))
        L2 = W.T @ J1
        J, P2 = _colwise_gs2(J1 - W @ L2, 0.0)
        L = L1 + L2 @ P1
        P = P2 @ P1
    else:
        L = np.zeros((0, m))
        J, P = _colwise_gs2(Up.copy(), tau)
    k = J.shape[1]
    Qm = np.zeros((r + k, r + m), dtype=np.float64)
    if r > 0:
        Qm[:r, :r] = np.diag(sigma)
        Qm[:r, r:] = L
    Qm[r:, r:] = P
    if Qm.shape[0] == 0:
        Vnew = np.zeros(((0 if V is None else V.shape[0]) + m, 0))
        return (np.zeros((n, 0)) if W is None else W[:, :0]), np.zeros(0), Vnew
    Ub, sb, Vbt = np.linalg.svd(Qm, full_matrices=False)
    keep = sb > eps_sv * sb[0] if sb.size and sb[0] > 0 else np.zeros(sb.shape, bool)
    keep[r_max:] = False
    Ub = Ub[:, keep]
    sb = sb[keep]
    Vb = Vbt.T[:, keep]
    basis = J if r == 0 else np.concatenate([W, J], axis=1)
    Wn = basis @ Ub
    p_rows = 0 if V is None else V.shape[0]
    Vn = np.zeros((p_rows + m, sb.shape[0]), dtype=np.float64)
    if r > 0:
        Vn[:p_rows] = V @ Vb[:r]
    Vn[p_rows:] = Vb[r:]
    Wn, _ = orthogonality_check(Wn, eps_svd)
    return Wn, sb, Vn


def orthogonality_check(W: np.ndarray, eps_svd: float) -> Tuple[np.ndarray, bool]:
    """Step 6: the orthogonality test at the end of Algorithm 2, read with an
    absolute value, |w_1^T w_r| > min(eps_svd, eps * N), and when it fires the
    re-orthogonalisation W = Q R (LAPACK Householder QR), with the signs of
    Q's columns chosen so that R has a positive diagonal: then column i of the
    result is the normalised part of w_i orthogonal to w_1 .. w_{i-1}, so no
    column changes orientation and W Sigma V^T moves only by the lost
    orthogonality.  Returns (W, fired)."""
    n, r = W.shape
    if r < 2 or not abs(W[:, 0] @ W[:, -1]) > min(eps_svd, EPS * n):
        return W, False
    Qf, Rf = np.linalg.qr(W)
    return Qf * np.where(np.diag(Rf) < 0, -1.0, 1.0), True


def pod_block_incremental(blocks: Sequence[np.ndarray], ns: int, nt: int, r_max: int,
                          eps_svd: float = 1e-12, eps_sv: float = 1e-14,
                          cols_per_update: Optional[int] = None) -> dict:
    """Block form of the incremental POD of Sec. 4.2, then the temporal
    bases of Eqs. incrementaltemporalsnapshotmat / temporalincrementalbasis.
    One update takes one parameter's Nt snapshots, or, with cols_per_update,
    that many consecutive columns of U = [U_1 ... U_nmu]; cols_per_update = 1
    streams the snapshots one at a time, the rank-one update of Algorithm 2."""
    if cols_per_update is None:
        parts = list(blocks)
    else:
        U = snapshot_matrix(blocks)
        parts = [U[:, c:c + cols_per_update] for c in range(0, U.shape[1], cols_per_update)]
    W = s = V = None
    for Up in parts:
        W, s, V = incremental_update(W, s, V, Up, r_max, eps_svd, eps_sv)
    n_mu = len(blocks)
    Nt = blocks[0].shape[1]
    T, tsv = temporal_bases(V, n_mu, Nt, ns, nt)
    return dict(W=W, sigma=s, V=V, Phi_s=W[:, :ns].copy(), T=T, temporal_sigma=tsv)


def canonical_signs(X: np.ndarray) -> np.ndarray:
    """Flip each column so that its entry of largest magnitude (lowest index
    on ties) is positive; singular vectors are defined up to sign."""
    X = np.array(X, dtype=np.float64, copy=True)
    if X.ndim == 1:
        X = X[:, None]
    idx = np.argmax(np.abs(X), axis=0)
    sgn = np.sign(X[idx, np.arange(X.shape[1])])
    sgn[sgn == 0] = 1.0
    return X * sgn
