"""Oracle: the learned surrogate mu -> uhat gated by the reduced space-time
residual.  The paper has no surrogate (its many-query motivation is the
future-work paragraph of Sec. 8); this FP64 restatement fixes what the GPU
kernels compute.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Network: x (2) -> Z1 = x W1^T + b1 -> H1 = gelu(Z1) -> Z2 = H1 W2^T + b2 ->
H2 = gelu(Z2) -> Y = H2 W3^T + b3 (n_out = ns*nt), with the exact GELU
gelu(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2.
Loss: mean squared error over the batch and the n_out outputs, against
targets normalised per component, (uhat - mean) / std.
Training: Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias correction), cosine
learning-rate decay over all steps, minibatches taken in the order of a
per-epoch affine permutation i -> (a i + b) mod n whose a, b come from
SplitMix64 (the counter-based generator of Steele, Lea and Flood) keyed by
(seed, epoch).
Gate: accept a prediction if ||Ahat^st uhat - rhs|| / ||rhs|| <= gate, else
solve the reduced system (Eq. st-galerkin).
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np
from scipy.special import erf

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)
MASK64 = (1 << 64) - 1


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / SQRT2))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / SQRT2)) + z * np.exp(-0.5 * z * z) * INV_SQRT_2PI


def forward(params, X):
    (W1, b1), (W2, b2), (W3, b3) = params
    Z1 = X @ W1.T + b1
    H1 = gelu(Z1)
    Z2 = H1 @ W2.T + b2
    H2 = gelu(Z2)
    Y = H2 @ W3.T + b3
    return Y, (X, Z1, H1, Z2, H2)


def loss_and_grads(params, X, T):
    """MSE loss and its gradients (manual backward through the network)."""
    (W1, b1), (W2, b2), (W3, b3) = params
    Y, (X, Z1, H1, Z2, H2) = forward(params, X)
    R = Y - T
    B, n_out = Y.shape
    loss = float(np.mean(R * R))
    dY = 2.0 * R / (B * n_out)
    dW3 = dY.T @ H2
    db3 = dY.sum(axis=0)
    dZ2 = (dY @ W3) * gelu_grad(Z2)
    dW2 = dZ2.T @ H1
    db2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ W2) * gelu_grad(Z1)
    dW1 = dZ1.T @ X
    db1 = dZ1.sum(axis=0)
    return loss, [(dW1, db1), (dW2, db2), (dW3, db3)]


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update with bias correction; state = (t, m, v), t counts steps."""
    t, m, v = state
    t += 1
    new_p, new_m, new_v = [], [], []
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        out = []
        for x, g, mm, vv in ((W, gW, mW, vW), (b, gb, mb, vb)):
            mm = beta1 * mm + (1 - beta1) * g
            vv = beta2 * vv + (1 - beta2) * g * g
            mh = mm / (1 - beta1 ** t)
            vh = vv / (1 - beta2 ** t)
            out.append((x - lr * mh / (np.sqrt(vh) + eps), mm, vv))
        new_p.append((out[0][0], out[1][0]))
        new_m.append((out[0][1], out[1][1]))
        new_v.append((out[0][2], out[1][2]))
    return new_p, (t, new_m, new_v)


def adam_init(params):
    z = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    return (0, z, [(np.zeros_like(W), np.zeros_like(b)) for W, b in params])


def cosine_lr(step: int, total: int, lr0: float) -> float:
    return 0.5 * lr0 * (1.0 + math.cos(math.pi * step / max(total, 1)))


def splitmix64(x: int) -> int:
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def epoch_permutation(n: int, seed: int, epoch: int) -> np.ndarray:
    """i -> (a i + b) mod n with gcd(a, n) = 1, a and b from SplitMix64."""
    a = splitmix64((seed + 2 * epoch) & MASK64) % n
    b = splitmix64((seed + 2 * epoch + 1) & MASK64) % n
    a = max(a, 1)
    while math.gcd(a, n) != 1:
        a = a + 1 if a + 1 < n else 1
    return (a * np.arange(n, dtype=np.int64) + b) % n


def target_stats(U: np.ndarray, floor: float = 1e-30) -> Tuple[np.ndarray, np.ndarray]:
    """Per-component mean and standard deviation of the training targets."""
    mean = U.mean(axis=0)
    std = np.sqrt(np.maximum(((U - mean) ** 2).mean(axis=0), floor))
    return mean, std


def train(params, X, T, epochs: int, batch: int, lr0: float, seed: int) -> Tuple[list, List[float]]:
    """FP64 replica of the training schedule (epochs of shuffled minibatches)."""
    n = X.shape[0]
    steps_per_epoch = (n + batch - 1) // batch
    total = epochs * steps_per_epoch
    state = adam_init(params)
    losses = []
    step = 0
    for e in range(epochs):
        perm = epoch_permutation(n, seed, e)
        acc = 0.0
        for j in range(steps_per_epoch):
            idx = perm[j * batch:(j + 1) * batch]
            loss, g = loss_and_grads(params, X[idx], T[idx])
            params, state = adam_step(params, g, state, cosine_lr(step, total, lr0))
            acc += loss * len(idx)
            step += 1
        losses.append(acc / n)
    return params, losses


def gate_residual(A: np.ndarray, rhs: np.ndarray, uhat: np.ndarray) -> float:
    """||Ahat^st uhat - rhs|| / ||rhs|| (the acceptance test of a prediction)."""
    return float(np.linalg.norm(A @ uhat - rhs) / np.linalg.norm(rhs))
