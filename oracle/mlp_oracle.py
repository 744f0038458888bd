"""FP64 CPU reference of the learned warm start's network -- TEST INFRASTRUCTURE ONLY.

The warm start proposes initial states for the QI search (it replaces rand_between of
Alg. 4): a per-site multilayer perceptron maps features of site i to a logit z_i of
P(s_i = +1). This module restates its definition in plain numpy FP64 so the CUDA kernels
(forward, backward, features) can be checked against it; only tests import it.

Features of site i (n spins, J symmetric with zero diagonal):
  f0 = h_i
  f1 = sum_j J_ij / sqrt(n)
  f2 = sum_j |J_ij| / n
  f3 = sqrt(sum_j J_ij^2 / n)
  f4 = max_{j != i} J_ij
  f5 = min_{j != i} J_ij
  f6 = sum_j J_ij h_j / sqrt(n)
  f7 = sum_j J_ij sign(h_j) / sqrt(n)          (sign(0) = 0)

Network (weights rounded to BF16, round-to-nearest-even, before use; biases FP32 values):
  a1 = X W1 + b1, h1 = relu(a1); a2 = h1 W2 + b2, h2 = relu(a2); a3 = h2 W3 + b3,
  h3 = relu(a3); z = h3 w4 + b4.
Loss: mean binary cross-entropy with labels y_i = 1 if s_i = +1 else 0:
  L = mean(softplus(z) - y z).
Gradients are taken with respect to the rounded weights (the master copy receives them).
"""
from __future__ import annotations

import numpy as np

N_FEATURES = 8


def features(J, h) -> np.ndarray:
    J = np.asarray(J, np.float64)
    h = np.asarray(h, np.float64)
    n = h.shape[0]
    off = ~np.eye(n, dtype=bool)
    Jm = np.where(off, J, np.nan)
    sh = np.sign(h)
    X = np.stack([
        h,
        J.sum(1) / np.sqrt(n),
        np.abs(J).sum(1) / n,
        np.sqrt((J * J).sum(1) / n),
        np.nanmax(Jm, 1),
        np.nanmin(Jm, 1),
        (J @ h) / np.sqrt(n),
        (J @ sh) / np.sqrt(n),
    ], axis=1)
    return X


def bf16(x) -> np.ndarray:
    """Round float32 values to the nearest BF16 (ties to even), returned as float64."""
    x32 = np.asarray(x, np.float32)
    u = x32.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)


def forward(params, X, round_weights=True):
    """params: dict W1 (F,H), b1 (H,), W2 (H,H), b2, W3 (H,H), b3, w4 (H,), b4 (scalar).
    round_weights=False uses the weights as given (for finite-difference checks)."""
    rnd = bf16 if round_weights else (lambda a: np.asarray(a, np.float64))
    W1, W2, W3, w4 = (rnd(params[k]) for k in ("W1", "W2", "W3", "w4"))
    b1, b2, b3 = (np.asarray(params[k], np.float64) for k in ("b1", "b2", "b3"))
    b4 = float(params["b4"])
    X = np.asarray(X, np.float64)
    a1 = X @ W1 + b1
    h1 = np.maximum(a1, 0)
    a2 = h1 @ W2 + b2
    h2 = np.maximum(a2, 0)
    a3 = h2 @ W3 + b3
    h3 = np.maximum(a3, 0)
    z = h3 @ w4 + b4
    return z, (X, a1, h1, a2, h2, a3, h3)


def loss_and_grad(params, X, y, round_weights=True):
    z, (X, a1, h1, a2, h2, a3, h3) = forward(params, X, round_weights)
    y = np.asarray(y, np.float64)
    M = z.shape[0]
    L = float(np.mean(np.logaddexp(0, z) - y * z))
    dz = (1.0 / (1.0 + np.exp(-z)) - y) / M
    rnd = bf16 if round_weights else (lambda a: np.asarray(a, np.float64))
    W2, W3, w4 = (rnd(params[k]) for k in ("W2", "W3", "w4"))
    g = {}
    g["w4"] = h3.T @ dz
    g["b4"] = dz.sum()
    da3 = np.outer(dz, w4) * (a3 > 0)
    g["W3"] = h2.T @ da3
    g["b3"] = da3.sum(0)
    da2 = (da3 @ W3.T) * (a2 > 0)
    g["W2"] = h1.T @ da2
    g["b2"] = da2.sum(0)
    da1 = (da2 @ W2.T) * (a1 > 0)
    g["W1"] = X.T @ da1
    g["b1"] = da1.sum(0)
    return L, g


PARAM_ORDER = ["W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4"]


def flatten(g) -> np.ndarray:
    return np.concatenate([np.asarray(g[k], np.float64).reshape(-1) for k in PARAM_ORDER])


def unflatten(v, F=N_FEATURES, H=256) -> dict:
    shapes = {"W1": (F, H), "b1": (H,), "W2": (H, H), "b2": (H,), "W3": (H, H), "b3": (H,), "w4": (H,), "b4": ()}
    out, o = {}, 0
    for k in PARAM_ORDER:
        sz = int(np.prod(shapes[k])) if shapes[k] else 1
        out[k] = np.asarray(v[o:o + sz], np.float64).reshape(shapes[k]) if shapes[k] else float(v[o])
        o += sz
    return out
