"""Oracle: space-time reduced operators, reduced solve and reconstruction
(Secs. 3.2 and 4.3).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Index conventions: reduced unknown (i, j) -> i + ns*j, i < ns spatial mode,
j < nt temporal mode (Eq. spacetimebasis); T (Nt x ns*nt) holds phi_t^{i,j}
in column i + ns*j; Phi_s is N x ns.

* ``spatial_reduced``  -- Ahat_q = Phi_s^T A_q Phi_s (reduced system matrix of
  Eq. galerkin, one per affine term).
* ``temporal_products`` -- the diagonal-block products of Eq. ij-block-matrix:
  G[(i',j'),(i,j)] = sum_k dt_k phi_{i'j'}[k] phi_{ij}[k],
  M_i[j',j] = sum_k phi_{ij'}[k] phi_{ij}[k],
  S_i[j',j] = sum_{k=1}^{Nt-1} phi_{ij'}[k+1] phi_{ij}[k].
* ``st_operator``      -- Ahat^st(mu) entrywise from those products:
  delta_{i'i} (M_i - S_i)[j',j] - Ahat(mu)[i',i] G[(i',j'),(i,j)].
* ``st_operator_literal`` -- the same blocks evaluated literally as
  sum_k (D_k^{j'} D_k^j - dt_k D_k^{j'} Ahat D_k^j) - sum_k D_{k+1}^{j'} D_k^j
  with the diagonal matrices D_k^j of Eq. temporaldiagonal.
* ``st_rhs``           -- fhat^st, block j = sum_k dt_k D_k^j Bhat f^k
  (Eq. j-block-vector).
* ``st_initial``       -- uhat0^st = Phi_st^T u0^st; from the definition of
  u0^st (Eq. ststate) block j is D_1^j Phi_s^T u0 for every j.  The printed
  Eq. first-block-initial-vector (block 1 = (sum_k D_k^1) uhat0, others 0)
  disagrees with that definition; ``st_initial_printed`` keeps the printed
  form for the test that shows the difference.
* ``st_basis``         -- explicit Phi_st, column i + ns*j = phi_t^{i,j} (x)
  phi_s^i (Eq. spacetimebasisvec), for brute-force checks on tiny inputs.
* ``solve``            -- Ahat^st uhat = fhat^st + uhat0^st (Eq. st-galerkin)
  by LAPACK partial-pivot LU (numpy.linalg.solve).
* ``reconstruct``      -- u^st ~= Phi_st uhat (Eq. ststateapproximation), by
  blocks: u^k = sum_{i,j} uhat_{ij} phi_t^{i,j}[k] phi_s^i.
* ``spatial_march``    -- the spatial Galerkin ROM of Sec. 3.1 (Eq. galerkin)
  marched by backward Euler (Eq. space_reduced_discretized_ODE) with the
  reference state 0: (I - dt_k Ahat) uhat^k = uhat^{k-1} + dt_k Bhat f^k,
  uhat^0 = Phi_s^T u0, one LAPACK solve per step.
* ``fom_residual``     -- r^k(u^k, u^{k-1}) = u^k - u^{k-1} - dt_k A u^k -
  dt_k B f^k (Eq. residual) for every step of a trajectory.
* ``spatial_error_bound`` -- the residual-based bound of Theorem 1,
  ||u^k - u~^k|| <= sum_{i<=k} (prod_{j=i..k} xi_j) ||r^i||, with
  xi_j = ||(I - dt_j A)^-1||_2, plus the term (prod_{j<=k} xi_j) ||u^0 - u~^0||
  that the one-step bound (Eq. one-timestep-bound) carries when u~^0 != u^0.
"""
from __future__ import annotations

from typing import Optional, Tuple

import numpy as np
import scipy.sparse as sp

from .fom import affine_operator


def spatial_reduced(rowptr, col, vals, Phi_s: np.ndarray) -> np.ndarray:
    """Ahat_q = Phi_s^T A_q Phi_s for each affine term q; shape (Q, ns, ns)."""
    Q = vals.shape[0]
    out = []
    for q in range(Q):
        e = np.zeros(Q)
        e[q] = 1.0
        Aq = affine_operator(rowptr, col, vals, e)
        out.append(Phi_s.T @ (Aq @ Phi_s))
    return np.array(out)


def temporal_products(T: np.ndarray, ns: int, nt: int, dt: np.ndarray
                      ) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    n = ns * nt
    G = T.T @ (dt[:, None] * T)
    M = np.zeros((ns, nt, nt))
    S = np.zeros((ns, nt, nt))
    for i in range(ns):
        Ti = T[:, [i + ns * j for j in range(nt)]]
        M[i] = Ti.T @ Ti
        S[i] = Ti[1:].T @ Ti[:-1]
    assert G.shape == (n, n)
    return G, M, S


def st_operator(Ahat_mu: np.ndarray, G: np.ndarray, M: np.ndarray, S: np.ndarray,
                ns: int, nt: int) -> np.ndarray:
    n = ns * nt
    A = np.zeros((n, n))
    for jp in range(nt):
        for j in range(nt):
            blk = -Ahat_mu * G[jp * ns:(jp + 1) * ns, j * ns:(j + 1) * ns]
            blk[np.arange(ns), np.arange(ns)] += M[:, jp, j] - S[:, jp, j]
            A[jp * ns:(jp + 1) * ns, j * ns:(j + 1) * ns] = blk
    return A


def _D(T: np.ndarray, ns: int, k: int, j: int) -> np.ndarray:
    """D_k^j = diag(phi_t^{1,j}[k], ..., phi_t^{ns,j}[k]) (Eq. temporaldiagonal)."""
    return np.diag(T[k, j * ns:(j + 1) * ns])


def st_operator_literal(Ahat_mu: np.ndarray, T: np.ndarray, dt: np.ndarray, ns: int,
                        nt: int) -> np.ndarray:
    Nt = T.shape[0]
    n = ns * nt
    A = np.zeros((n, n))
    for jp in range(nt):
        for j in range(nt):
            blk = np.zeros((ns, ns))
            for k in range(Nt):
                Dp = _D(T, ns, k, jp)
                Dj = _D(T, ns, k, j)
                blk += Dp @ Dj - dt[k] * (Dp @ Ahat_mu @ Dj)
            for k in range(Nt - 1):
                blk -= _D(T, ns, k + 1, jp) @ _D(T, ns, k, j)
            A[jp * ns:(jp + 1) * ns, j * ns:(j + 1) * ns] = blk
    return A


def st_rhs(Phi_s: np.ndarray, T: np.ndarray, B: np.ndarray, F: np.ndarray, dt: np.ndarray,
           ns: int, nt: int) -> np.ndarray:
    Bhat = Phi_s.T @ B                    # reduced input matrix (Eq. galerkin)
    Nt = T.shape[0]
    f = np.zeros(ns * nt)
    for j in range(nt):
        acc = np.zeros(ns)
        for k in range(Nt):
            acc += dt[k] * (T[k, j * ns:(j + 1) * ns] * (Bhat @ F[k]))
        f[j * ns:(j + 1) * ns] = acc
    return f


def st_initial(Phi_s: np.ndarray, T: np.ndarray, u0: Optional[np.ndarray], ns: int,
               nt: int) -> np.ndarray:
    if u0 is None:
        return np.zeros(ns * nt)
    u0hat = Phi_s.T @ u0
    return np.concatenate([T[0, j * ns:(j + 1) * ns] * u0hat for j in range(nt)])


def st_initial_printed(Phi_s: np.ndarray, T: np.ndarray, u0: np.ndarray, ns: int,
                       nt: int) -> np.ndarray:
    out = np.zeros(ns * nt)
    out[:ns] = T[:, :ns].sum(axis=0) * (Phi_s.T @ u0)
    return out


def st_basis(Phi_s: np.ndarray, T: np.ndarray, ns: int, nt: int) -> np.ndarray:
    N = Phi_s.shape[0]
    Nt = T.shape[0]
    out = np.zeros((N * Nt, ns * nt))
    for j in range(nt):
        for i in range(ns):
            out[:, i + ns * j] = np.kron(T[:, i + ns * j], Phi_s[:, i])
    return out


def sub_indices(ns_m: int, nt_m: int, ns: int) -> np.ndarray:
    """Indices (in the full i + ns*j ordering) of the nested sub-basis
    i < ns_m, j < nt_m, listed in the sub-basis order i + ns_m*j."""
    return np.array([i + ns * j for j in range(nt_m) for i in range(ns_m)], dtype=np.int64)


class ReducedModel:
    """Pre-computed reduced operators (offline phase of Sec. 4.3)."""

    def __init__(self, prob, Phi_s: np.ndarray, T: np.ndarray, ns: int, nt: int):
        self.ns, self.nt = ns, nt
        self.Phi_s, self.T = Phi_s, T
        self.Ahat_q = spatial_reduced(prob.rowptr, prob.col, prob.vals, Phi_s)
        self.G, self.M, self.S = temporal_products(T, ns, nt, prob.dt)
        self.fhat = st_rhs(Phi_s, T, prob.B, prob.F, prob.dt, ns, nt)
        self.u0hat = st_initial(Phi_s, T, prob.u0, ns, nt)
        # spatial ROM operators (Eq. galerkin): Bhat, uhat0 = Phi_s^T u0
        self.Bhat = Phi_s.T @ prob.B
        self.u0s = np.zeros(ns) if prob.u0 is None else Phi_s.T @ prob.u0
        self.dt, self.F = prob.dt, prob.F

    def Ahat(self, theta: np.ndarray) -> np.ndarray:
        return np.tensordot(theta, self.Ahat_q, axes=(0, 0))

    def operator(self, theta: np.ndarray, ns_m: Optional[int] = None,
                 nt_m: Optional[int] = None) -> Tuple[np.ndarray, np.ndarray]:
        """(Ahat^st, fhat^st + uhat0^st) of the nested (ns_m, nt_m) sub-model."""
        ns_m = self.ns if ns_m is None else ns_m
        nt_m = self.nt if nt_m is None else nt_m
        full = st_operator(self.Ahat(theta), self.G, self.M, self.S, self.ns, self.nt)
        idx = sub_indices(ns_m, nt_m, self.ns)
        return full[np.ix_(idx, idx)], (self.fhat + self.u0hat)[idx]

    def solve(self, theta: np.ndarray, ns_m: Optional[int] = None,
              nt_m: Optional[int] = None) -> np.ndarray:
        A, f = self.operator(theta, ns_m, nt_m)
        return np.linalg.solve(A, f)

    def spatial_march(self, theta: np.ndarray, ns_m: Optional[int] = None) -> np.ndarray:
        """Spatial-ROM trajectory (ns_m x Nt) on the leading ns_m modes."""
        ns_m = self.ns if ns_m is None else ns_m
        return spatial_march(self.Ahat(theta)[:ns_m, :ns_m], self.Bhat[:ns_m], self.F, self.dt,
                             self.u0s[:ns_m])

    def reconstruct(self, uhat: np.ndarray, ns_m: Optional[int] = None,
                    nt_m: Optional[int] = None) -> np.ndarray:
        ns_m = self.ns if ns_m is None else ns_m
        nt_m = self.nt if nt_m is None else nt_m
        return reconstruct(self.Phi_s, self.T, uhat, self.ns, ns_m, nt_m)


def reconstruct(Phi_s: np.ndarray, T: np.ndarray, uhat: np.ndarray, ns: int, ns_m: int,
                nt_m: int) -> np.ndarray:
    """U (N x Nt) with u^k = sum_{i<ns_m, j<nt_m} uhat[i + ns_m j] phi_t^{ij}[k] phi_s^i."""
    Nt = T.shape[0]
    C = np.zeros((ns_m, Nt))
    for j in range(nt_m):
        for i in range(ns_m):
            C[i] += uhat[i + ns_m * j] * T[:, i + ns * j]
    return Phi_s[:, :ns_m] @ C


def rel_error(U_ref: np.ndarray, U: np.ndarray) -> float:
    """Global space-time relative error ||U_ref - U||_F / ||U_ref||_F."""
    return float(np.linalg.norm(U_ref - U) / np.linalg.norm(U_ref))


def st_inf_norm(U: np.ndarray) -> float:
    """Space-time infinity norm max_k ||u^k||_2 (Eq. spacetimeinfnorm)."""
    return float(np.max(np.linalg.norm(U, axis=0)))


def spatial_march(Ahat_mu: np.ndarray, Bhat: np.ndarray, F: np.ndarray, dt: np.ndarray,
                  uhat0: Optional[np.ndarray] = None) -> np.ndarray:
    """Backward-Euler march of the spatial ROM (Eq. space_reduced_discretized_ODE,
    reference state 0).  Returns Uhat (ns x Nt) whose column k-1 is uhat^k."""
    ns = Ahat_mu.shape[0]
    u = np.zeros(ns) if uhat0 is None else np.array(uhat0, dtype=np.float64)
    out = np.empty((ns, dt.shape[0]))
    for k in range(dt.shape[0]):
        u = np.linalg.solve(np.eye(ns) - dt[k] * Ahat_mu, u + dt[k] * (Bhat @ F[k]))
        out[:, k] = u
    return out


def fom_residual(A, dt: np.ndarray, B: np.ndarray, F: np.ndarray, U: np.ndarray,
                 u_init: np.ndarray) -> np.ndarray:
    """Columns r^k(u^k, u^{k-1}) (Eq. residual) of a trajectory U (N x Nt)
    started from u_init."""
    R = np.empty_like(U)
    prev = u_init
    for k in range(dt.shape[0]):
        R[:, k] = U[:, k] - prev - dt[k] * (A @ U[:, k]) - dt[k] * (B @ F[k])
        prev = U[:, k]
    return R


def spatial_error_bound(A, dt: np.ndarray, R: np.ndarray, e0: float = 0.0) -> np.ndarray:
    """Right-hand side of Theorem 1 at every step k = 1..Nt for residual
    columns R (N x Nt); xi_j from the dense SVD of I - dt_j A (small cases)."""
    n = A.shape[0]
    Ad = A.toarray() if sp.issparse(A) else np.asarray(A)
    xi = np.array([1.0 / np.linalg.svd(np.eye(n) - h * Ad, compute_uv=False).min() for h in dt])
    rn = np.linalg.norm(R, axis=0)
    out = np.empty(dt.shape[0])
    for k in range(dt.shape[0]):
        b = np.prod(xi[:k + 1]) * e0
        for i in range(k + 1):
            b += np.prod(xi[i:k + 1]) * rn[i]
        out[k] = b
    return out
