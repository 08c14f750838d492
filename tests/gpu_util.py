"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

from oracle import fom, pod, strom


def torch_mod():
    import torch
    return torch


def dev_tensor(a, dtype=None):
    torch = torch_mod()
    t = torch.tensor(np.ascontiguousarray(a), device="cuda:0")
    return t if dtype is None else t.to(dtype)


def make_model(p, **opts):
    import paper_1910_01260_gb300 as st
    torch = torch_mod()
    return st.Model(p.rowptr, p.col, p.vals, st.options(**opts),
                    stream=torch.cuda.current_stream().cuda_stream)


def dev_B(p):
    # column-major N x n_in on the device = row-major (n_in, N)
    return dev_tensor(p.B.T.copy())


def gpu_fom(m, p, mus, Nt=None, u0=None, F=None, dt=None, with_iters=False):
    """Returns (list of N x Nt snapshot blocks, status, iters)."""
    torch = torch_mod()
    Nt = p.Nt if Nt is None else Nt
    dt = p.dt[:Nt] if dt is None else dt
    F = p.F[:Nt] if F is None else F
    n = len(mus)
    snaps = torch.full((n, Nt, p.N), float("nan"), dtype=torch.float64, device="cuda:0")
    status = torch.full((n,), -1, dtype=torch.int32, device="cuda:0")
    iters = torch.zeros((Nt, n), dtype=torch.int32, device="cuda:0") if with_iters else None
    u0d = None if u0 is None else dev_tensor(u0)
    m.st_fom_march(p.theta(np.asarray(mus)), dt, u0d, dev_B(p), F, snaps, iters, status)
    torch.cuda.synchronize()
    S = snaps.cpu().numpy()
    blocks = [S[k].T.copy() for k in range(n)]
    return blocks, status.cpu().numpy(), (iters.cpu().numpy() if with_iters else None)


def oracle_fom(p, mus, Nt=None, u0=None):
    Nt = p.Nt if Nt is None else Nt
    out = []
    for mu in mus:
        A = fom.affine_operator(p.rowptr, p.col, p.vals, p.theta(mu))
        out.append(fom.fom_march(A, p.dt[:Nt], p.B, p.F[:Nt], u0))
    return out


def rel_max(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def projector_dist(A, B):
    return float(np.abs(A @ A.T - B @ B.T).max())


def _oracle_fom_one(args):
    name, k, Nt = args
    from workloads import problem_for
    p = problem_for(name)
    A = fom.affine_operator(p.rowptr, p.col, p.vals, p.theta(p.train_mu[k]))
    return fom.fom_march(A, p.dt[:Nt], p.B, p.F[:Nt], None)


def oracle_fom_train_parallel(name, Nt=None, procs=None):
    """The oracle's snapshot blocks of every training parameter of a named
    workload, one process per parameter (spawned, so safe after CUDA use)."""
    import multiprocessing as mp
    import os
    from workloads import problem_for
    p = problem_for(name)
    Nt = p.Nt if Nt is None else Nt
    procs = procs or min(len(p.train_mu), os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_oracle_fom_one, [(name, k, Nt) for k in range(len(p.train_mu))])
