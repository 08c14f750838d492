"""Oracle: full-order model (FOM) of the parametric LTI system (Sec. 2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``affine_operator``  -- A(mu) = sum_q theta_q A_q (problem statement, Eq.
  Dynamicalstate, with the affine split of the transport workloads).
* ``fom_march``        -- backward Euler, one linear solve per step (Eq. fom):
  (I - dt_k A) u^k = u^{k-1} + dt_k B f^k, t_k = sum_{j<=k} dt_j.  The
  default per-step solve is a direct sparse LU (the plain definition of the
  step); ``solver="bicgstab"`` runs textbook BiCGSTAB, and ``"dense"`` uses
  numpy.linalg.solve for tiny cases.
* ``st_fom_system``    -- the all-at-once space-time system A^st u^st =
  f^st + u0^st (Eqs. st-fom, stsystemmat, ststate): block lower bidiagonal,
  diagonal blocks I - dt_k A, sub-diagonal blocks -I.
"""
from __future__ import annotations

from typing import Dict, Optional, Tuple

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def affine_operator(rowptr: np.ndarray, col: np.ndarray, vals: np.ndarray,
                    theta: np.ndarray) -> sp.csr_matrix:
    """A(mu) = sum_q theta_q A_q as a CSR matrix (all terms share one pattern)."""
    n = rowptr.shape[0] - 1
    v = np.tensordot(np.asarray(theta, dtype=np.float64), vals, axes=(0, 0))
    return sp.csr_matrix((v, col.astype(np.int64), rowptr), shape=(n, n))


def bicgstab(K, b: np.ndarray, x0: np.ndarray, tol: float = 1e-14, maxit: int = 1000
             ) -> Tuple[np.ndarray, int, str]:
    """Unpreconditioned BiCGSTAB (van der Vorst), shadow residual r^ = r_0,
    stopping at ||r|| <= tol * ||b||.  Returns (x, iterations, status) with
    status in {"ok", "not_converged", "breakdown"}."""
    x = x0.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, "ok"
    r = b - K @ x
    if np.linalg.norm(r) <= tol * bnorm:
        return x, 0, "ok"
    rhat = r.copy()
    rho_old = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    for it in range(1, maxit + 1):
        rho = rhat @ r
        if abs(rho) < 1e-300:
            return x, it, "breakdown"
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = K @ p
        alpha = rho / (rhat @ v)
        s = r - alpha * v
        if np.linalg.norm(s) <= tol * bnorm:
            x = x + alpha * p
            return x, it, "ok"
        t = K @ s
        tt = t @ t
        if tt == 0.0:
            return x, it, "breakdown"
        omega = (t @ s) / tt
        x = x + alpha * p + omega * s
        r = s - omega * t
        if np.linalg.norm(r) <= tol * bnorm:
            return x, it, "ok"
        if abs(omega) < 1e-300:
            return x, it, "breakdown"
        rho_old = rho
    return x, maxit, "not_converged"


def fom_march(A: sp.csr_matrix, dt: np.ndarray, B: np.ndarray, F: np.ndarray,
              u0: Optional[np.ndarray] = None, solver: str = "splu", tol: float = 1e-14,
              maxit: int = 2000, iters: Optional[list] = None, x0_order: int = 0) -> np.ndarray:
    """Backward-Euler march of Eq. fom.  Returns U (N x Nt) whose column k-1
    is u^k (Eq. snapshotmat uses the same column order).

    x0_order (BiCGSTAB only) picks the initial iterate of each step: the
    polynomial of degree o = min(k, x0_order) through the last o + 1 levels,
    evaluated one step ahead (0: the previous level).  It changes the
    iteration count, not the solution beyond the stopping tolerance."""
    n = A.shape[0]
    nt_steps = dt.shape[0]
    u = np.zeros(n) if u0 is None else np.asarray(u0, dtype=np.float64).copy()
    levels = [u.copy()]
    U = np.empty((n, nt_steps), dtype=np.float64)
    eye = sp.identity(n, format="csc")
    cache: Dict[float, object] = {}
    for k in range(nt_steps):
        h = float(dt[k])
        rhs = u + h * (B @ F[k])
        if solver == "splu":
            if h not in cache:
                cache[h] = spla.splu((eye - h * A).tocsc())
            u = cache[h].solve(rhs)
        elif solver == "dense":
            K = np.eye(n) - h * A.toarray()
            u = np.linalg.solve(K, rhs)
        elif solver == "bicgstab":
            K = (eye - h * A).tocsr()
            o = min(k, x0_order)
            x0 = np.zeros(n)
            for i in range(o + 1):
                x0 += (-1) ** i * math.comb(o + 1, i + 1) * levels[-1 - i]
            u, it, st = bicgstab(K, rhs, x0, tol=tol, maxit=maxit)
            if st != "ok":
                raise RuntimeError(f"oracle BiCGSTAB {st} at step {k + 1}")
            if iters is not None:
                iters.append(it)
        else:
            raise ValueError(solver)
        U[:, k] = u
        levels = (levels + [u.copy()])[-(x0_order + 1):]
    return U


def st_fom_system(A: sp.csr_matrix, dt: np.ndarray, B: np.ndarray, F: np.ndarray,
                  u0: Optional[np.ndarray] = None) -> Tuple[sp.csr_matrix, np.ndarray]:
    """A^st and f^st + u0^st of Eqs. stsystemmat / ststate (time-major blocks,
    u^st = [u^1; ...; u^Nt])."""
    n = A.shape[0]
    nt_steps = dt.shape[0]
    eye = sp.identity(n, format="csr")
    blocks = [[None] * nt_steps for _ in range(nt_steps)]
    for k in range(nt_steps):
        blocks[k][k] = eye - dt[k] * A
        if k > 0:
            blocks[k][k - 1] = -eye
    Ast = sp.bmat(blocks, format="csr")
    rhs = np.concatenate([dt[k] * (B @ F[k]) for k in range(nt_steps)])
    if u0 is not None:
        rhs[:n] += u0
    return Ast, rhs


def st_fom_solve(A: sp.csr_matrix, dt: np.ndarray, B: np.ndarray, F: np.ndarray,
                 u0: Optional[np.ndarray] = None) -> np.ndarray:
    """Solve the space-time FOM all at once (tiny cases); returns U (N x Nt)."""
    Ast, rhs = st_fom_system(A, dt, B, F, u0)
    ust = spla.spsolve(Ast.tocsc(), rhs)
    return ust.reshape(dt.shape[0], A.shape[0]).T.copy()
