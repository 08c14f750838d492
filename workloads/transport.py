"""Synthetic linear kinetic-transport workloads (one energy group, isotropic
scattering, discrete ordinates, first-order upwind finite differences) written
as the parametric LTI system of Sec. 2:

    du/dt = A(mu) u + B f(t),   u(0) = u0,

with A(mu) = V (L^+ Sigma_s L - H) in the isotropic one-group reduction of
Sec. 6 (Eqs. Lnmdef, Lnm+def, Hdef, DAE): H = C_l + Sigma_t per direction,
the scattering source is "take the scalar-flux moment, then broadcast", and
v = 1.  The paper's SCB spatial discretisation is replaced by cell-centred
upwind differences on the unit square/segment with vacuum inflow (Eq. dirbcs).

The operator is split into three affine terms sharing one sparsity pattern,
A(mu) = sum_q theta_q(mu) A_q with theta(mu) = (1, mu1, mu1*mu2):
  A_0 = -v D_Omega            (streaming, parameter independent)
  A_1 = -v diag(rho)          (total cross-section sigma_t = mu1 * rho)
  A_2 = +v diag(rho) P        (scattering sigma_s = mu2 * sigma_t, P = 1_L w^T (x) I)
where rho is a seeded base field.  Unknowns are direction-major,
idx = l * n_cells + cell, cells x-fastest (Sec. 6.2 zone ordering).

This module is input generation only; it contains no step of the reduced
order method.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Dict, List, Optional, Tuple

import numpy as np

# ---------------------------------------------------------------------------
# Angular quadrature (Sec. 6.2, Carlson-Lathrop level-symmetric sets with
# L = nu (nu + 2) directions, weights normalised so that sum w = 1 because the
# paper normalises the unit-sphere measure to one).
# ---------------------------------------------------------------------------


def gauss_legendre_1d(n: int) -> Tuple[np.ndarray, np.ndarray]:
    """n-point Gauss-Legendre directions on [-1, 1] for slab geometry.

    Returns (mu, w) with sum(w) = 1 (the Legendre weights halved)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return x.astype(np.float64), (0.5 * w).astype(np.float64)


# First direction cosine of the standard level-symmetric sets.
_LS_MU1 = {4: 0.3500212, 6: 0.2666355}


def level_symmetric_2d(nu: int) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Level-symmetric S_nu set (nu in {4, 6}) restricted to the upper
    hemisphere (xi > 0) and projected onto (mu, eta).

    Levels: mu_i^2 = mu_1^2 + (i-1) * Delta with Delta = 2 (1 - 3 mu_1^2)/(nu-2);
    directions of an octant are (mu_i, mu_j, mu_k) with i + j + k = nu/2 + 2.
    Weights are per permutation class, solved from the zeroth and fourth
    moment conditions of one octant (sum w = 1, sum w mu^4 = 1/5); the second
    moment 1/3 then holds by the permutation symmetry of each class.
    Returns (mu, eta, w), sum w = 1, L = nu (nu + 2) / 2 directions."""
    if nu not in _LS_MU1:
        raise ValueError("only S4 and S6 are tabulated")
    mu1 = _LS_MU1[nu]
    half = nu // 2
    delta = 2.0 * (1.0 - 3.0 * mu1 * mu1) / (nu - 2)
    levels = np.sqrt(mu1 * mu1 + delta * np.arange(half))
    trip = [(i, j, k) for i in range(1, half + 1) for j in range(1, half + 1)
            for k in range(1, half + 1) if i + j + k == half + 2]
    classes: Dict[Tuple[int, ...], List[Tuple[int, int, int]]] = {}
    for t in trip:
        classes.setdefault(tuple(sorted(t)), []).append(t)
    keys = sorted(classes)
    # moment equations for the class weights (one octant, total weight 1)
    ncls = len(keys)
    if ncls > 2:
        raise ValueError("more weight classes than moment conditions")
    rows = np.array([[len(classes[c]) for c in keys],
                     [sum(levels[t[0] - 1] ** 4 for t in classes[c]) for c in keys]],
                    dtype=np.float64)[:ncls]
    rhs = np.array([1.0, 1.0 / 5.0], dtype=np.float64)[:ncls]
    wc = np.linalg.solve(rows, rhs)
    octant = []
    for ci, c in enumerate(keys):
        for t in classes[c]:
            octant.append((levels[t[0] - 1], levels[t[1] - 1], wc[ci]))
    mus, etas, ws = [], [], []
    for sx in (1.0, -1.0):
        for sy in (1.0, -1.0):
            for (a, b, wt) in octant:
                mus.append(sx * a)
                etas.append(sy * b)
                ws.append(wt)
    w = np.array(ws, dtype=np.float64)
    w /= w.sum()
    return np.array(mus, dtype=np.float64), np.array(etas, dtype=np.float64), w


# ---------------------------------------------------------------------------
# Problem container
# ---------------------------------------------------------------------------


@dataclasses.dataclass
class Problem:
    name: str
    dim: int
    M: int                      # cells per axis
    n_cells: int
    L: int                      # number of directions
    N: int                      # spatial unknowns = L * n_cells
    mu_dir: np.ndarray          # direction cosines (x)
    eta_dir: np.ndarray         # direction cosines (y), zeros in 1-D
    w: np.ndarray               # quadrature weights, sum = 1
    rho: np.ndarray             # base cross-section field per cell
    rowptr: np.ndarray          # int64 [N + 1]
    col: np.ndarray             # int32 [nnz], sorted within rows
    vals: np.ndarray            # float64 [Q, nnz], affine terms A_q
    B: np.ndarray               # float64 [N, n_in], input matrix (column major use)
    F: np.ndarray               # float64 [Nt, n_in], input samples f^k at t_k
    dt: np.ndarray              # float64 [Nt]
    u0: np.ndarray              # float64 [N]
    Nt: int
    T: float
    mu_lo: np.ndarray           # parameter box lower corner (mu1, mu2)
    mu_hi: np.ndarray           # parameter box upper corner
    train_mu: np.ndarray        # [n_train, 2]
    test_mu: np.ndarray         # [n_test, 2]
    ns: int
    nt: int

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    @property
    def Q(self) -> int:
        return int(self.vals.shape[0])

    @property
    def n_in(self) -> int:
        return int(self.B.shape[1])

    def theta(self, mu: np.ndarray) -> np.ndarray:
        return theta_of_mu(mu)


def theta_of_mu(mu: np.ndarray) -> np.ndarray:
    """Affine coefficients theta(mu) = (1, mu1, mu1 * mu2), shape [..., 3]."""
    mu = np.asarray(mu, dtype=np.float64)
    one = np.ones(mu.shape[:-1], dtype=np.float64)
    return np.stack([one, mu[..., 0], mu[..., 0] * mu[..., 1]], axis=-1)


def train_grid(n1: int, n2: int, lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """Tensor grid at the mid-point quantiles (2i+1)/(2n); mu1 is the outer
    index, so sample p = i1 * n2 + i2."""
    q1 = (2 * np.arange(n1) + 1) / (2.0 * n1)
    q2 = (2 * np.arange(n2) + 1) / (2.0 * n2)
    g1 = lo[0] + q1 * (hi[0] - lo[0])
    g2 = lo[1] + q2 * (hi[1] - lo[1])
    return np.array([[a, b] for a in g1 for b in g2], dtype=np.float64)


def uniform_mu(n: int, lo: np.ndarray, hi: np.ndarray, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return lo + rng.random((n, 2)) * (hi - lo)


# ---------------------------------------------------------------------------
# Sparse operator terms
# ---------------------------------------------------------------------------


def _build_terms(dim: int, M: int, mu_d: np.ndarray, eta_d: np.ndarray, w: np.ndarray,
                 rho: np.ndarray, v: float, streaming: bool):
    L = w.shape[0]
    nc = M ** dim
    N = L * nc
    h = 1.0 / M
    rows = np.arange(N, dtype=np.int64)
    ell = rows // nc
    cell = rows % nc
    ix = cell % M
    nslot = L + dim
    cols = np.empty((N, nslot), dtype=np.int64)
    a0 = np.zeros((N, nslot), dtype=np.float64)
    a1 = np.zeros((N, nslot), dtype=np.float64)
    a2 = np.zeros((N, nslot), dtype=np.float64)
    valid = np.ones((N, nslot), dtype=bool)
    rho_c = rho[cell]
    for lp in range(L):
        cols[:, lp] = lp * nc + cell
        a2[:, lp] = v * rho_c * w[lp]
    on_diag = (np.arange(L)[None, :] == ell[:, None])
    a1[:, :L] = np.where(on_diag, -v * rho_c[:, None], 0.0)
    mu_l = mu_d[ell]
    eta_l = eta_d[ell]
    if streaming:
        dcoef = -v * (np.abs(mu_l) / h + (np.abs(eta_l) / h if dim == 2 else 0.0))
        a0[:, :L] = np.where(on_diag, dcoef[:, None], 0.0)
        # x upwind neighbour
        step = np.where(mu_l > 0, -1, 1)
        nb = ix + step
        ok = (nb >= 0) & (nb < M) & (mu_l != 0)
        cols[:, L] = ell * nc + cell + step
        a0[:, L] = v * np.abs(mu_l) / h
        valid[:, L] = ok
        if dim == 2:
            iy = cell // M
            stepy = np.where(eta_l > 0, -1, 1)
            nby = iy + stepy
            oky = (nby >= 0) & (nby < M) & (eta_l != 0)
            cols[:, L + 1] = ell * nc + cell + stepy * M
            a0[:, L + 1] = v * np.abs(eta_l) / h
            valid[:, L + 1] = oky
    else:
        valid[:, L:] = False
        cols[:, L:] = 0
    sentinel = np.int64(N + 1)
    ckey = np.where(valid, cols, sentinel)
    order = np.argsort(ckey, axis=1, kind="stable")
    ckey = np.take_along_axis(ckey, order, axis=1)
    vs = [np.take_along_axis(a, order, axis=1) for a in (a0, a1, a2)]
    keep = ckey != sentinel
    counts = keep.sum(axis=1)
    rowptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    col = ckey[keep].astype(np.int32)
    vals = np.stack([a[keep] for a in vs], axis=0)
    return N, nc, rowptr, col, vals


def _rho_field(dim: int, M: int, kind: str) -> np.ndarray:
    if kind == "homogeneous":
        return np.ones(M ** dim, dtype=np.float64)
    if dim == 1:
        return np.random.default_rng(0).uniform(0.5, 2.0, M)
    rng = np.random.default_rng(1)
    xs, ys = rng.uniform(0.25, 0.75, 2)
    vals = rng.uniform(0.5, 5.0, 4)
    xc = (np.arange(M) + 0.5) / M
    X, Y = np.meshgrid(xc, xc, indexing="xy")  # X[iy, ix]
    region = (X > xs).astype(int) + 2 * (Y > ys).astype(int)
    return vals[region].reshape(-1)  # cell = ix + M * iy


def _source(dim: int, M: int, kind: str) -> np.ndarray:
    xc = (np.arange(M) + 0.5) / M
    if kind == "box":
        q = np.zeros(M)
        q[24 * M // 64: 40 * M // 64] = 1.0
        return q if dim == 1 else np.outer(q, q).reshape(-1)
    if kind == "gaussian":
        X, Y = np.meshgrid(xc, xc, indexing="xy")
        return np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2) / (2 * 0.1 ** 2)).reshape(-1)
    if kind == "none":
        return np.zeros(M ** dim)
    raise ValueError(kind)


def _g(kind: str) -> Callable[[np.ndarray, float], np.ndarray]:
    if kind == "sin":
        return lambda t, T: np.sin(np.pi * t / T)
    if kind == "ramp":
        return lambda t, T: t / T
    if kind == "const":
        return lambda t, T: np.ones_like(t)
    raise ValueError(kind)


def make_problem(name: str = "custom", dim: int = 1, M: int = 8, quad: str = "gl4",
                 Nt: int = 6, T: float = 1.0, rho: str = "seeded", source: str = "box",
                 g: str = "sin", u0: str = "zero", streaming: bool = True, v: float = 1.0,
                 mu_lo=(0.5, 0.1), mu_hi=(1.5, 0.9), train=(2, 2), n_test: int = 4,
                 ns: int = 4, nt: int = 2) -> Problem:
    """Generic builder; the named configurations below call it."""
    if quad.startswith("gl"):
        mu_d, w = gauss_legendre_1d(int(quad[2:]))
        eta_d = np.zeros_like(mu_d)
        if dim != 1:
            raise ValueError("Gauss-Legendre directions are for slab geometry")
    elif quad in ("s4", "s6"):
        mu_d, eta_d, w = level_symmetric_2d(int(quad[1:]))
        if dim != 2:
            raise ValueError("level-symmetric sets are used in 2-D")
    else:
        raise ValueError(quad)
    rho_f = _rho_field(dim, M, "homogeneous" if rho == "homogeneous" else "seeded")
    N, nc, rowptr, col, vals = _build_terms(dim, M, mu_d, eta_d, w, rho_f, v, streaming)
    L = w.shape[0]
    q = _source(dim, M, source)
    B = np.tile(v * q, L).reshape(N, 1).astype(np.float64)
    dt = np.full(Nt, T / Nt, dtype=np.float64)
    tk = np.cumsum(dt)
    F = _g(g)(tk, T).reshape(Nt, 1).astype(np.float64)
    if u0 == "zero":
        u0v = np.zeros(N, dtype=np.float64)
    elif u0 == "seeded":
        u0v = np.random.default_rng(3).uniform(0.0, 1.0, N)
    elif u0 == "isotropic":
        base = np.random.default_rng(3).uniform(0.0, 1.0, nc)
        u0v = np.tile(base, L)
    else:
        raise ValueError(u0)
    lo = np.array(mu_lo, dtype=np.float64)
    hi = np.array(mu_hi, dtype=np.float64)
    return Problem(name=name, dim=dim, M=M, n_cells=nc, L=L, N=N, mu_dir=mu_d, eta_dir=eta_d,
                   w=w, rho=rho_f, rowptr=rowptr, col=col, vals=vals, B=B, F=F, dt=dt, u0=u0v,
                   Nt=Nt, T=T, mu_lo=lo, mu_hi=hi, train_mu=train_grid(train[0], train[1], lo, hi),
                   test_mu=uniform_mu(n_test, lo, hi, 2), ns=ns, nt=nt)


# Named workloads: c1 a 1-D slab (64 cells, 8 Gauss directions, 50 steps, 2x2
# training parameters); c2 2-D S4 transport on 64x64 cells (N = 49,152, 200
# steps, 4x4 training parameters); c3 2-D S6 transport on 256x256 cells
# (N = 1,572,864, 500 steps, 8x4 training parameters); c4 c2's full-order
# model and training set with a basis built to (ns, nt) = (40, 12), for the
# 4096-parameter online batch; c5 the same model, for the surrogate.
CONFIGS: Dict[str, dict] = {
    "c1": dict(dim=1, M=64, quad="gl8", Nt=50, source="box", g="sin", mu_hi=(1.5, 0.9),
               train=(2, 2), n_test=8, ns=8, nt=4),
    "c2": dict(dim=2, M=64, quad="s4", Nt=200, source="gaussian", g="ramp", mu_hi=(1.5, 0.95),
               train=(4, 4), n_test=8, ns=20, nt=8),
    "c3": dict(dim=2, M=256, quad="s6", Nt=500, source="gaussian", g="ramp", mu_hi=(1.5, 0.95),
               train=(8, 4), n_test=4, ns=40, nt=12),
    "c4": dict(dim=2, M=64, quad="s4", Nt=200, source="gaussian", g="ramp", mu_hi=(1.5, 0.95),
               train=(4, 4), n_test=8, ns=40, nt=12),
}
CONFIGS["c5"] = dict(CONFIGS["c4"])

# Uneven reduced sizes of the batched online phase.
C4_SIZES = np.array([(10, 4), (20, 8), (30, 10), (40, 12)], dtype=np.int32)


def problem_for(name: str, **overrides) -> Problem:
    kw = dict(CONFIGS[name])
    kw.update(overrides)
    return make_problem(name=name, **kw)


def c4_batch(n: int = 4096, prob: Optional[Problem] = None, seed: int = 4):
    """Seeded online batch: parameters uniform in the box and reduced sizes
    drawn uniformly from C4_SIZES.  Returns (mu [n,2], ns_nt [n,2] int32)."""
    lo = np.array([0.5, 0.1]) if prob is None else prob.mu_lo
    hi = np.array([1.5, 0.95]) if prob is None else prob.mu_hi
    rng = np.random.default_rng(seed)
    mu = lo + rng.random((n, 2)) * (hi - lo)
    idx = rng.integers(0, len(C4_SIZES), n)
    return mu.astype(np.float64), C4_SIZES[idx].copy()


def c5_samples(n_train: int = 8192, n_infer: int = 65536, prob: Optional[Problem] = None):
    lo = np.array([0.5, 0.1]) if prob is None else prob.mu_lo
    hi = np.array([1.5, 0.95]) if prob is None else prob.mu_hi
    return uniform_mu(n_train, lo, hi, 5), uniform_mu(n_infer, lo, hi, 6)


# ---------------------------------------------------------------------------
# Surrogate network inputs: seeded initial weights and the mapping of mu to
# the network input.  (Random draws of the method are inputs to both sides.)
# ---------------------------------------------------------------------------

MLP_HIDDEN = 256


def mlp_init(n_out: int, hidden: int = MLP_HIDDEN, n_in: int = 2, seed: int = 5):
    """Kaiming-uniform weights (bound sqrt(6 / fan_in)) and zero biases for
    the 3-layer network n_in -> hidden -> hidden -> n_out.  Returns a list of
    (W [out x in], b [out]) float64 arrays."""
    rng = np.random.default_rng(seed)
    dims = [n_in, hidden, hidden, n_out]
    out = []
    for a, b in zip(dims[:-1], dims[1:]):
        bound = math.sqrt(6.0 / a)
        out.append((rng.uniform(-bound, bound, (b, a)), np.zeros(b)))
    return out


def mu_to_input(mu: np.ndarray, lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """Affine map of the parameter box onto [-1, 1]^2."""
    return 2.0 * (np.asarray(mu) - lo) / (hi - lo) - 1.0
