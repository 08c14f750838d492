"""Seeded synthetic inputs shared by the oracle and the GPU path.

Nothing in this package performs any step of the space-time reduced-order
method: it only builds the problem data -- affine operator terms A_q in CSR
form, the input matrix B, the input samples f^k, time steps, initial state and
parameter samples -- that both sides consume.
"""
from .transport import (  # noqa: F401
    CONFIGS,
    Problem,
    gauss_legendre_1d,
    level_symmetric_2d,
    make_problem,
    problem_for,
    theta_of_mu,
    train_grid,
    uniform_mu,
    c4_batch,
    c5_samples,
    mlp_init,
    mu_to_input,
)
