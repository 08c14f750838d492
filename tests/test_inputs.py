"""Pins of the seeded input generator (quadrature, operator terms, sizes)."""
import json
import os

import numpy as np
import pytest

from workloads import gauss_legendre_1d, level_symmetric_2d, make_problem, problem_for, theta_of_mu
from workloads.transport import C4_SIZES, c4_batch

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("kind", ["gl8", "s4", "s6"])
def test_quadrature_moments(kind):
    # Sec. 6.1 normalises the unit-sphere measure to one; an even-moment exact
    # set then integrates mu^2 to 1/3 and mu^4 to 1/5.
    if kind == "gl8":
        mu, w = gauss_legendre_1d(8)
        eta = None
        tol4 = 1e-14
    else:
        mu, eta, w = level_symmetric_2d(int(kind[1:]))
        tol4 = 1e-6 if kind == "s4" else 1e-14   # S4's mu_1 is tabulated to 7 digits
    assert w.min() > 0
    assert abs(w.sum() - 1) < 1e-14
    assert abs((w * mu).sum()) < 1e-14
    assert abs((w * mu ** 2).sum() - 1 / 3) < 1e-13
    assert abs((w * mu ** 4).sum() - 1 / 5) < tol4
    if eta is not None:
        assert abs((w * eta ** 2).sum() - 1 / 3) < 1e-13
        assert np.all(mu ** 2 + eta ** 2 < 1)       # projections of unit vectors with xi > 0
        assert abs((w * mu ** 2 * eta ** 2).sum() - 1 / 15) < 1e-6


def test_direction_counts_against_paper_sizes():
    # Sec. 6.2: L = nu (nu + 2) directions; Sec. 7 prints the resulting DOF.
    g = json.load(open(os.path.join(GOLDEN, "paper_sizes.json")))
    for ex in ("ex1", "ex2"):
        e = g[ex]
        nu = 8
        assert nu * (nu + 2) == e["directions"]
        zones = int(np.prod(e["mesh"]))
        dof = zones * e["directions"] * e["groups"]
        assert dof == e["dof_space"]
        assert dof * int(round(e["T_ns"] / e["dt_ns"])) == e["dof_spacetime"]
    # our one-group 2-D sets keep the xi > 0 half of the 3-D set
    assert level_symmetric_2d(4)[2].size == 4 * 6 // 2
    assert level_symmetric_2d(6)[2].size == 6 * 8 // 2


@pytest.mark.parametrize("name,N,nnz_row", [("c1", 512, 9), ("c2", 49152, 14)])
def test_config_sizes(name, N, nnz_row):
    p = problem_for(name)
    assert p.N == N
    counts = np.diff(p.rowptr)
    assert counts.max() == nnz_row
    assert p.vals.shape == (3, p.nnz)
    # columns sorted and unique within rows
    for r in range(0, p.N, max(1, p.N // 97)):
        c = p.col[p.rowptr[r]:p.rowptr[r + 1]]
        assert np.all(np.diff(c) > 0)


def _dense_terms(p):
    out = []
    for q in range(3):
        A = np.zeros((p.N, p.N))
        for r in range(p.N):
            for k in range(p.rowptr[r], p.rowptr[r + 1]):
                A[r, p.col[k]] += p.vals[q, k]
        out.append(A)
    return out


def test_operator_terms_structure():
    p = make_problem(dim=2, M=4, quad="s4", Nt=3)
    A0, A1, A2 = _dense_terms(p)
    nc = p.n_cells
    one = np.ones(p.N)
    # upwind streaming annihilates constants away from inflow boundaries
    y = A0 @ one
    for ell in range(p.L):
        for cell in range(nc):
            ix, iy = cell % p.M, cell // p.M
            inflow_x = (ix == 0) if p.mu_dir[ell] > 0 else (ix == p.M - 1)
            inflow_y = (iy == 0) if p.eta_dir[ell] > 0 else (iy == p.M - 1)
            if not inflow_x and not inflow_y:
                assert abs(y[ell * nc + cell]) < 1e-12
            else:
                assert y[ell * nc + cell] < 0
    # total cross-section term is -v rho on the diagonal
    assert np.allclose(A1, -np.diag(np.tile(p.rho, p.L)))
    # scattering: moment then broadcast, rows sum to v rho sum(w) = v rho
    assert np.allclose(A2 @ one, np.tile(p.rho, p.L))
    # every direction sees the same scalar flux: rank of A2 is n_cells
    assert np.linalg.matrix_rank(A2) == nc


def test_theta_and_batches():
    th = theta_of_mu(np.array([[2.0, 0.5], [1.0, 0.25]]))
    assert np.allclose(th, [[1, 2, 1], [1, 1, 0.25]])
    mu, sz = c4_batch(4096)
    assert mu.shape == (4096, 2) and sz.shape == (4096, 2)
    assert set(map(tuple, sz)) <= set(map(tuple, C4_SIZES))
    mu2, sz2 = c4_batch(4096)
    assert np.array_equal(mu, mu2) and np.array_equal(sz, sz2)   # seeded
