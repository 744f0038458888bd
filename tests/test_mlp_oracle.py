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


def test_row_statistics_f2_f3_on_a_hand_computed_instance():
    """f2 = sum_j |J_ij| / n and f3 = sqrt(sum_j J_ij^2 / n) on a 4-spin instance whose row values
    are chosen so the results are exact: row 0 = (0, 3, -4, 0) gives 7/4 and sqrt(25/4) = 5/2."""
    J = np.zeros((4, 4))
    for (i, j, v) in [(0, 1, 3.0), (0, 2, -4.0), (1, 2, 1.0), (1, 3, -2.0), (2, 3, 0.5)]:
        J[i, j] = J[j, i] = v
    h = np.array([1.0, -2.0, 0.0, 0.5])
    X = M.features(J, h)
    assert X[0, 2] == 7.0 / 4.0 and X[0, 3] == 2.5
    # row 1 = (3, 0, 1, -2): |.| sum 6, squares 14
    assert X[1, 2] == 6.0 / 4.0 and X[1, 3] == np.sqrt(14.0 / 4.0)
    # row 3 = (0, -2, 0.5, 0): the remaining features as written out by hand
    assert X[3, 0] == 0.5
    assert X[3, 1] == -1.5 / 2.0                       # sum_j J_3j / sqrt(4)
    assert X[3, 4] == 0.5 and X[3, 5] == -2.0          # max and min over j != 3 (the diagonal excluded)
    assert X[3, 6] == (-2.0 * -2.0 + 0.5 * 0.0) / 2.0  # sum_j J_3j h_j / sqrt(4)
    assert X[3, 7] == (-2.0 * -1.0 + 0.5 * 0.0) / 2.0  # sign(h_2) = sign(0) = 0
    # row 2 has no positive off-diagonal coupling but a zero diagonal: max over j != 2 is 1
    assert X[2, 4] == 1.0 and X[2, 5] == -4.0


def _tiny_net():
    """A 2-unit network whose every weight is a BF16 value, so rounding leaves it unchanged."""
    W1 = np.zeros((8, 2))
    W1[0] = [1.0, -1.0]
    W1[1] = [0.5, 0.25]
    return {"W1": W1, "b1": np.array([0.0, -1.0]), "W2": np.array([[1.0, -2.0], [3.0, 4.0]]),
            "b2": np.array([0.5, 0.0]), "W3": np.array([[2.0, 0.0], [0.0, 1.0]]), "b3": np.array([-1.0, 1.0]),
            "w4": np.array([0.5, -3.0]), "b4": 0.25}


def test_forward_of_a_hand_built_network():
    """z written out layer by layer by hand. Row 0: a1 = (2, -1.5) -> h1 = (2, 0); a2 = (2.5, -4)
    -> h2 = (2.5, 0); a3 = (4, 1) -> h3 = (4, 1); z = 0.5*4 - 3*1 + 0.25 = -0.75 (negative: no
    ReLU on the output). Row 1, X = (-1, 4): a1 = (1, 1) -> h1 = (1, 1); a2 = (4.5, 2); h3 from
    a3 = (2*4.5 - 1, 2 + 1) = (8, 3); z = 4 - 9 + 0.25 = -4.75. Row 2, X = (-3, 0): a1 = (-3, 2)
    -> h1 = (0, 2); a2 = (6.5, 8); a3 = (12, 9); z = 6 - 27 + 0.25 = -20.75."""
    X = np.zeros((3, 8))
    X[0, :2] = [1.0, 2.0]
    X[1, :2] = [-1.0, 4.0]
    X[2, :2] = [-3.0, 0.0]
    z, _ = M.forward(_tiny_net(), X)
    assert np.array_equal(z, [-0.75, -4.75, -20.75])


def test_forward_relu_zeroes_negative_preactivations_and_weights_are_rounded():
    p = _tiny_net()
    p["b3"] = np.array([-20.0, 1.0])      # row 0: a3 = (5 - 20, 1) -> h3 = (0, 1); z = -3 + 0.25
    X = np.zeros((1, 8))
    X[0, :2] = [1.0, 2.0]
    z, _ = M.forward(p, X)
    assert z[0] == -2.75
    # a weight between two BF16 values is rounded to the nearer one before use: 1 + 2^-10 -> 1
    p = _tiny_net()
    p["W3"] = np.array([[2.0 + 2.0 ** -9, 0.0], [0.0, 1.0 + 2.0 ** -10]])
    X = np.zeros((2, 8))
    X[0, :2] = [1.0, 2.0]                 # h2 = (2.5, 0)
    X[1, :2] = [-1.0, 4.0]                # h2 = (4.5, 2)
    z, _ = M.forward(p, X)
    assert np.array_equal(z, [-0.75, -4.75])
    z, _ = M.forward(p, X, round_weights=False)
    assert z[0] == 0.5 * (2.5 * (2.0 + 2.0 ** -9) - 1.0) - 3.0 * 1.0 + 0.25
    assert z[1] == 0.5 * (4.5 * (2.0 + 2.0 ** -9) - 1.0) - 3.0 * (2.0 * (1.0 + 2.0 ** -10) + 1.0) + 0.25


def test_loss_is_the_mean_binary_cross_entropy():
    """L = mean(log(1 + e^z) - y z) for the hand-built network's logits (-0.75, -4.75, -20.75)."""
    X = np.zeros((3, 8))
    X[0, :2] = [1.0, 2.0]
    X[1, :2] = [-1.0, 4.0]
    X[2, :2] = [-3.0, 0.0]
    y = np.array([1.0, 0.0, 1.0])
    L, _ = M.loss_and_grad(_tiny_net(), X, y)
    want = (np.log1p(np.exp(-0.75)) + 0.75 + np.log1p(np.exp(-4.75)) + np.log1p(np.exp(-20.75)) + 20.75) / 3
    assert L == pytest.approx(want, rel=1e-14)
