"""GPU parity of the learned surrogate and its residual gate against the FP64
oracle (oracle/mlp.py), on the 1-D slab model (ns*nt = 32 outputs).

Tolerances: the GPU network multiplies BF16 copies of weights and of the
hidden activations (8-bit mantissas, relative rounding 2^-9) with FP32
accumulation; three layers of such products give ~1e-2 relative deviation
from FP64, so gradients are compared at 3e-2 of each tensor's largest entry
and the loss at 2e-2.  The gate residual is evaluated in FP32 (relative
rounding 6e-8 on sums of 32 terms): 1e-5 relative."""
import numpy as np
import pytest

from gpu_util import dev_B, dev_tensor, make_model, oracle_fom, rel_max
from oracle import mlp, pod, strom
from workloads import mlp_init, mu_to_input, problem_for, uniform_mu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c1():
    p = problem_for("c1")
    blocks = oracle_fom(p, p.train_mu)
    ref = pod.pod_exact(blocks, p.ns, p.nt)
    rm = strom.ReducedModel(p, ref["Phi_s"], ref["T"], p.ns, p.nt)
    mu = uniform_mu(512, p.mu_lo, p.mu_hi, 11)
    U = np.array([rm.solve(p.theta(x)) for x in mu])
    return p, ref, rm, mu, U


def _model(p, ref):
    m = make_model(p)
    m.st_model_set_basis(p.ns, p.nt, p.Nt, dev_tensor(ref["Phi_s"].T.copy()), dev_tensor(ref["T"].T.copy()))
    m.st_rom_assemble(p.dt, dev_B(p), p.F, None)
    return m


def _flat(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params]).astype(np.float32)


def _unflat(v, shapes):
    out, o = [], 0
    for (a, b) in shapes:
        W = v[o:o + a * b].reshape(a, b)
        o += a * b
        bias = v[o:o + a]
        o += a
        out.append((W, bias))
    return out


def test_loss_and_gradients_match_oracle(c1):
    p, ref, rm, mu, U = c1
    m = _model(p, ref)
    init = mlp_init(p.ns * p.nt, hidden=256)
    flat = _flat(init)
    n = 256
    loss, g = m.st_rom_surrogate_loss_grad(n, dev_tensor(mu[:n]), p.mu_lo, p.mu_hi, dev_tensor(U[:n]), flat)
    # oracle at the same (FP32-rounded) parameters and batch
    params = [(W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)) for W, b in init]
    X = mu_to_input(mu[:n], p.mu_lo, p.mu_hi)
    mean, std = mlp.target_stats(U[:n])
    l_ref, g_ref = mlp.loss_and_grads(params, X, (U[:n] - mean) / std)
    assert abs(loss - l_ref) < 2e-2 * l_ref
    shapes = [(W.shape[0], W.shape[1]) for W, _ in init]
    for (gW, gb), (rW, rb) in zip(_unflat(g, shapes), g_ref):
        assert np.abs(gW - rW).max() < 3e-2 * np.abs(rW).max()
        assert np.abs(gb - rb).max() < 3e-2 * max(np.abs(rb).max(), 1e-30)
    m.close()


def test_training_follows_the_oracle_schedule(c1):
    p, ref, rm, mu, U = c1
    m = _model(p, ref)
    init = mlp_init(p.ns * p.nt, hidden=256)
    n, epochs, batch, lr = 512, 40, 128, 2e-3
    losses = m.st_rom_surrogate_train(n, dev_tensor(mu), p.mu_lo, p.mu_hi, dev_tensor(U), init=_flat(init),
                                      epochs=epochs, batch=batch, lr=lr, seed=5)
    X = mu_to_input(mu, p.mu_lo, p.mu_hi)
    mean, std = mlp.target_stats(U)
    params = [(W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)) for W, b in init]
    _, l_ref = mlp.train(params, X, (U - mean) / std, epochs=epochs, batch=batch, lr0=lr, seed=5)
    l_ref = np.array(l_ref)
    assert losses[-1] < 0.05 * losses[0]
    # same schedule and data order: the BF16 run tracks the FP64 one
    assert np.all(np.abs(losses[:5] - l_ref[:5]) < 0.05 * l_ref[:5])
    assert losses[-1] < 3.0 * l_ref[-1] + 1e-4
    m.close()


def test_gate_residual_and_fallback(c1):
    torch = __import__("torch")
    p, ref, rm, mu, U = c1
    m = _model(p, ref)
    n_out = p.ns * p.nt
    init = mlp_init(n_out, hidden=256)
    # last layer zero, bias t: every prediction is mean + std * t, known to the oracle
    t = np.random.default_rng(3).standard_normal(n_out) * 0.01
    init[2] = (np.zeros_like(init[2][0]), t)
    m.st_rom_surrogate_train(len(mu), dev_tensor(mu), p.mu_lo, p.mu_hi, dev_tensor(U), init=_flat(init), epochs=0,
                             batch=64)
    mean, std = mlp.target_stats(U)
    pred = mean + std * t.astype(np.float32).astype(np.float64)
    q_mu = uniform_mu(300, p.mu_lo, p.mu_hi, 12)
    th = p.theta(q_mu)
    gates = []
    for x in th:
        A, rhs = rm.operator(x)
        gates.append(mlp.gate_residual(A, rhs, pred))
    gates = np.array(gates)
    gate = float(np.median(gates))
    n = len(q_mu)
    uhat = torch.zeros((n, n_out), dtype=torch.float64, device="cuda:0")
    res = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    used = torch.full((n,), -1, dtype=torch.int32, device="cuda:0")
    nf = m.st_rom_surrogate_infer(n, dev_tensor(q_mu), dev_tensor(th), gate, uhat, res, used)
    torch.cuda.synchronize()
    uh, rr, us = uhat.cpu().numpy(), res.cpu().numpy(), used.cpu().numpy()
    assert nf == int(us.sum())
    clear = np.abs(gates - gate) > 1e-4 * gate
    assert np.array_equal(us[clear], (gates[clear] > gate).astype(np.int32))
    for k in range(n):
        if us[k] == 0:
            # the gate's products are FP32-accurate (tensor-core FP32 sums of
            # three-part BF16 splits): ~2^-23 of ||Ahat^st x|| ~ ||rhs|| here
            assert abs(rr[k] - gates[k]) < 1e-5 * gates[k] + 4e-7
            assert rel_max(uh[k], pred) < 1e-6
        else:
            want = rm.solve(th[k])
            assert rel_max(uh[k], want) < 1e-10 and rr[k] < 1e-12
    m.close()


def test_trained_surrogate_accuracy(c1):
    torch = __import__("torch")
    p, ref, rm, mu, U = c1
    m = _model(p, ref)
    m.st_rom_surrogate_train(len(mu), dev_tensor(mu), p.mu_lo, p.mu_hi, dev_tensor(U), epochs=300, batch=128,
                             lr=2e-3, seed=5)
    q_mu = uniform_mu(200, p.mu_lo, p.mu_hi, 13)
    th = p.theta(q_mu)
    n, n_out = len(q_mu), p.ns * p.nt
    uhat = torch.zeros((n, n_out), dtype=torch.float64, device="cuda:0")
    res = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    used = torch.zeros(n, dtype=torch.int32, device="cuda:0")
    m.st_rom_surrogate_infer(n, dev_tensor(q_mu), dev_tensor(th), 1e30, uhat, res, used)
    torch.cuda.synchronize()
    uh = uhat.cpu().numpy()
    errs = [np.linalg.norm(uh[k] - rm.solve(th[k])) / np.linalg.norm(rm.solve(th[k])) for k in range(n)]
    assert np.median(errs) < 2e-2
    m.close()
