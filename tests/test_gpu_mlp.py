"""Learned warm start on the GPU: features, forward, gradients and training kernels against
the FP64 reference (oracle/mlp_oracle.py), and the warm-started search against the oracle."""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from oracle import oracle as O
from paper_2010_00180_gb300 import build, inputs as I, qis

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    qis.load()


def test_features_match_reference():
    net = qis.MLP(hidden=64, max_sites=4096, batch=256, max_n=300)
    for ens, n in (("gaussian", 300), ("pm1", 97)):
        J, h = I.instance(ens, n, seed=n)
        got = net.features(J, h)
        want = M.features(J, h).astype(np.float32)
        np.testing.assert_allclose(got, want, rtol=2e-6, atol=1e-6)


def test_forward_and_gradients_match_fp64_reference():
    H, F = 256, 8
    net = qis.MLP(hidden=H, max_sites=4096, batch=512, max_n=64, seed=5)
    p = M.unflatten(net.get_params().astype(np.float64), F, H)
    rng = np.random.default_rng(0)
    X = rng.normal(0, 1, (512, F)).astype(np.float32)
    y = (rng.random(512) < 0.4).astype(np.float32)
    z = net.forward(X)
    z_ref, _ = M.forward(p, X)
    np.testing.assert_allclose(z, z_ref, rtol=1e-4, atol=1e-4 * np.abs(z_ref).max())
    L, g = net.loss_grad(X, y)
    L_ref, g_ref = M.loss_and_grad(p, X, y)
    assert abs(L - L_ref) <= 1e-5 * abs(L_ref)
    gv = M.flatten(g_ref)
    o = 0
    for k in M.PARAM_ORDER:
        sz = np.asarray(g_ref[k]).size
        a, b = g[o:o + sz].astype(np.float64), gv[o:o + sz]
        np.testing.assert_allclose(a, b, rtol=2e-3, atol=2e-4 * max(np.abs(b).max(), 1e-12), err_msg=k)
        o += sz


def best_states(J, h, K=30, R=8, iters=30):
    n = h.shape[0]
    ctx = qis.Context(K=K, R=R, precision="split_bf16", max_n=n)
    ctx.create_instance(J, h)
    ctx.init_states(0, I.random_states(n, R, seed=77))
    ctx.iterate(iters)
    out = ctx.topk_states(0, 1)
    ctx.close()
    return out["bits"][0]


def test_training_and_warm_started_search():
    n, n_train = 64, 48
    net = qis.MLP(hidden=256, max_sites=n * n_train, batch=1024, max_n=n, seed=1)
    for k in range(n_train):
        J, h = I.instance("gaussian", n, seed=500, inst=k)
        net.add_example(J, h, best_states(J, h))
    first = net.train(1, lr=1e-3)
    last = net.train(30, lr=1e-3)
    assert last < first
    # warm start of held-out instances: search 0 starts from sign(z), every search then
    # follows Alg. 3 exactly as the oracle does from the same initial state
    K, R, iters = 20, 4, 15
    ctx = qis.Context(K=K, R=R, precision="split_bf16", max_n=n, max_instances=2)
    starts = []
    for k in range(2):
        J, h = I.instance("gaussian", n, seed=900, inst=k)
        ctx.create_instance(J, h)
        ctx.init_states_learned(k, net)
        z = net.forward(net.features(J, h))
        starts.append([ctx.search_list(k, r)["bits"][0] for r in range(R)])
        assert np.array_equal(I.unpack_bits(starts[k][0], n)[0], (z < 0).astype(np.uint8))
        assert len({tuple(s) for s in starts[k]}) > 1          # the draws differ from the argmax
    ctx.iterate(iters)
    for k in range(2):
        J, h = I.instance("gaussian", n, seed=900, inst=k)
        for r in range(R):
            ref = O.qi_search(J, h, K, iters, starts[k][r])
            got = ctx.search_list(k, r)
            assert np.array_equal(got["bits"], ref["bits"][: ref["count"]])
            assert np.array_equal(got["E"], ref["E"][: ref["count"]])


def test_learned_initial_states_are_lower_than_random():
    """What the network gains: the energy of its proposed initial states against random ones
    on held-out instances (the search-time comparison is in bench.py's warm-start workload)."""
    n, n_train, R = 100, 64, 16
    net = qis.MLP(hidden=256, max_sites=n * n_train, batch=2048, max_n=n, seed=2)
    for k in range(n_train):
        J, h = I.instance("gaussian", n, seed=600, inst=k)
        net.add_example(J, h, best_states(J, h))
    net.train(40, lr=1e-3)
    e_learned, e_random = [], []
    for k in range(8):
        J, h = I.instance("gaussian", n, seed=700, inst=k)
        ctx = qis.Context(K=8, R=R, precision="split_bf16", max_n=n)
        ctx.create_instance(J, h)
        ctx.init_states_learned(0, net)
        e_learned += [ctx.search_list(0, r)["E"][0] for r in range(R)]
        ctx.init_states(0, I.random_states(n, R, seed=701, inst=k))
        e_random += [ctx.search_list(0, r)["E"][0] for r in range(R)]
        ctx.close()
    print(f"mean initial energy: learned {np.mean(e_learned):.2f}, random {np.mean(e_random):.2f}")
    assert np.mean(e_learned) < np.mean(e_random)


def test_adam_steps_match_numpy():
    """Two training steps on a one-batch training set against Adam written out in numpy (beta
    0.9 / 0.999, eps 1e-8, bias-corrected moments, the FP32 master weights updated), each step's
    gradient taken from the library's own backward pass at the weights of that step."""
    n, lr = 200, 1e-3
    net = qis.MLP(hidden=32, max_sites=1024, batch=1024, max_n=n, seed=9)
    J, h = I.instance("gaussian", n, seed=810)
    bits = I.random_states(n, 1, seed=811)[0]
    net.add_example(J, h, bits)
    X = net.features(J, h)
    y = (I.unpack_bits(bits, n)[0] == 0).astype(np.float32)   # y_i = 1 <=> s_i = +1 (sigma_i = 0)
    p = net.get_params().astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    b1, b2, eps = 0.9, 0.999, 1e-8
    for t in (1, 2):
        _, g = net.loss_grad(X, y)
        g = g.astype(np.float64)
        net.train(1, lr=lr)                         # one batch: one Adam step
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        p = p - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
        got = net.get_params().astype(np.float64)
        # FP32 arithmetic in the kernel and atomics in the gradient sums: each update agrees to a
        # small fraction of the step size lr
        np.testing.assert_allclose(got, p, rtol=0, atol=2e-3 * lr + 1e-7, err_msg=f"step {t}")
        p = got                                     # continue from the library's weights
