"""Pins of the FP64 reference of the warm-start network (oracle/mlp_oracle.py)."""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_2010_00180_gb300 import inputs as I


def random_params(F=8, H=32, seed=0):
    rng = np.random.default_rng(seed)
    return {"W1": rng.normal(0, 0.5, (F, H)), "b1": rng.normal(0, 0.1, H), "W2": rng.normal(0, 0.3, (H, H)),
            "b2": rng.normal(0, 0.1, H), "W3": rng.normal(0, 0.3, (H, H)), "b3": rng.normal(0, 0.1, H),
            "w4": rng.normal(0, 0.3, H), "b4": 0.1}


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(1).normal(0, 3, 10000).astype(np.float32)
    x[:4] = [1.0, -0.0, 3.14159, 1e-30]
    want = torch.tensor(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16(x), want)


def test_features_definition():
    J, h = I.instance("gaussian", 30, seed=3)
    X = M.features(J, h)
    n = 30
    i = 7
    row = np.delete(J[i], i)
    assert X[i, 0] == h[i]
    assert np.isclose(X[i, 1], J[i].sum() / np.sqrt(n))
    assert X[i, 4] == row.max() and X[i, 5] == row.min()
    assert np.isclose(X[i, 6], (J[i] * h).sum() / np.sqrt(n))
    assert np.isclose(X[i, 7], (J[i] * np.sign(h)).sum() / np.sqrt(n))


def test_backward_matches_central_differences():
    """The analytic gradient against central differences of the FP64 loss. Weights are made
    BF16 values first, so rounding them is the identity and the rounded network is the
    smooth function being differentiated."""
    H = 16
    p = random_params(H=H, seed=2)
    for k in ("W1", "W2", "W3", "w4"):
        p[k] = M.bf16(p[k])
    rng = np.random.default_rng(3)
    X = rng.normal(0, 1, (40, 8))
    y = (rng.random(40) < 0.5).astype(float)
    L, g = M.loss_and_grad(p, X, y)
    L2, g2 = M.loss_and_grad(p, X, y, round_weights=False)
    assert L == L2 and np.array_equal(M.flatten(g), M.flatten(g2))
    gv = M.flatten(g)
    v = M.flatten(p)
    eps = 1e-6
    for idx in range(0, v.size, 3):
        vp, vm = v.copy(), v.copy()
        vp[idx] += eps
        vm[idx] -= eps
        Lp, _ = M.loss_and_grad(M.unflatten(vp, 8, H), X, y, round_weights=False)
        Lm, _ = M.loss_and_grad(M.unflatten(vm, 8, H), X, y, round_weights=False)
        fd = (Lp - Lm) / (2 * eps)
        assert abs(fd - gv[idx]) <= 1e-6 + 1e-5 * abs(gv[idx]), (idx, fd, gv[idx])
