"""Flip-set variants on the GPU (single flips only; spin exchanges only) against the oracle:
every search's list after each iteration, the Alg. 4 merge, a sector smaller than the list,
the candidate counters, and a config-3-sized exchange run on sampled searches."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2010_00180_gb300 import build, inputs as I, qis

pytestmark = pytest.mark.gpu

VARIANTS = [("single", 1), ("exchange", 2)]
MODES = [("split_bf16", "gaussian"), ("fp64", "gaussian"), ("pm1_fp8", "pm1")]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    qis.load()


def same(g, o, what=""):
    c = o["count"]
    assert g["count"] == c, what
    for key in ("bits", "E", "used", "stamp"):
        assert np.array_equal(g[key], o[key][:c]), (what, key)


@pytest.mark.parametrize("name,fl", VARIANTS)
@pytest.mark.parametrize("prec,ens", MODES)
def test_every_iteration_matches_oracle(name, fl, prec, ens):
    n, K, R, iters = 70, 20, 4, 15
    J, h = I.instance(ens, n, seed=200, inst=fl)
    phi = I.random_states(n, R, seed=201, inst=fl)
    ctx = qis.Context(K=K, R=R, precision=prec, max_n=n, flips=name)
    ctx.create_instance(J, h)
    ctx.init_states(0, phi)
    for t in range(1, iters + 1):
        ctx.iterate(1)
        for r in range(R):
            same(ctx.search_list(0, r), O.qi_search(J, h, K, t, phi[r], flips=fl), f"t={t} r={r}")
    ctx.close()


@pytest.mark.parametrize("name,fl", VARIANTS)
@pytest.mark.parametrize("prec,ens", MODES)
def test_many_instances_and_merge(name, fl, prec, ens):
    ns, K, R, iters = [130, 97, 64], 40, 6, 30
    ctx = qis.Context(K=K, R=R, precision=prec, max_n=max(ns), max_instances=len(ns), flips=name)
    data = []
    for k, n in enumerate(ns):
        J, h = I.instance(ens, n, seed=210, inst=k)
        phi = I.random_states(n, R, seed=211, inst=k)
        ctx.create_instance(J, h)
        ctx.init_states(k, phi)
        data.append((J, h, phi))
    ctx.iterate(iters)
    for k, (J, h, phi) in enumerate(data):
        for r in range(R):
            same(ctx.search_list(k, r), O.qi_search(J, h, K, iters, phi[r], flips=fl), f"inst={k} r={r}")
        got = ctx.topk_states(k, K + 1)
        ref = O.qi_multi_search(J, h, K, iters, phi, flips=fl)
        assert got["count"] == ref["count"]
        assert np.array_equal(got["bits"], ref["bits"][: ref["count"]])
        assert np.array_equal(got["src"], ref["src"][: ref["count"]])
        np.testing.assert_allclose(got["E"], ref["E"][: ref["count"]], rtol=1e-9)
    ctx.close()


@pytest.mark.parametrize("prec,ens", MODES)
def test_exchange_sector_smaller_than_list(prec, ens):
    """Two up spins in n = 9: a sector of 36 states, K + 1 = 50 slots."""
    n, K, R, iters = 9, 49, 3, 60
    J, h = I.instance(ens, n, seed=220)
    phi = np.array([[(1 << 1) | (1 << 6)], [(1 << 0) | (1 << 8)], [(1 << 3) | (1 << 4)]], np.uint64)
    ctx = qis.Context(K=K, R=R, precision=prec, max_n=n, flips="exchange")
    ctx.create_instance(J, h)
    ctx.init_states(0, phi)
    ctx.iterate(iters)
    for r in range(R):
        ref = O.qi_search(J, h, K, iters, phi[r], flips=2)
        assert ref["count"] == 36
        same(ctx.search_list(0, r), ref, f"r={r}")
    ctx.close()


@pytest.mark.parametrize("prec,ens", MODES)
def test_exchange_skewed_magnetisation(prec, ens):
    """Few up spins (1, 3, 6 of 200) or few down spins: the bound's subset draws low-a sites
    from each spin class, so it keeps enough up-down pairs however the spins are split."""
    n, K, iters = 200, 40, 25
    J, h = I.instance(ens, n, seed=225)
    rng = np.random.default_rng(226)
    rows = []
    for m in (1, 3, 6, n - 1, n - 4):
        x = np.zeros(n, np.uint8)
        x[rng.choice(n, m, replace=False)] = 1
        rows.append(I.pack_bits(x[None, :])[0])
    phi = np.stack(rows)
    ctx = qis.Context(K=K, R=len(rows), precision=prec, max_n=n, flips="exchange")
    ctx.create_instance(J, h)
    ctx.init_states(0, phi)
    for t in range(1, iters + 1):
        ctx.iterate(1)
        if t % 5 == 0:
            for r in range(len(rows)):
                same(ctx.search_list(0, r), O.qi_search(J, h, K, t, phi[r], flips=2), f"t={t} r={r}")
    ctx.close()


def test_candidate_counters_follow_the_flip_set():
    n, K, R, iters = 50, 30, 4, 12
    J, h = I.instance("gaussian", n, seed=230)
    phi = I.random_states(n, R, seed=231)
    for name, fl in [("single_pair", 0)] + VARIANTS:
        ctx = qis.Context(K=K, R=R, precision="split_bf16", max_n=n, flips=name)
        ctx.create_instance(J, h)
        ctx.init_states(0, phi)
        ctx.iterate(iters)
        pairs, singles = ctx.candidate_count()
        want_p = want_s = 0
        for r in range(R):
            prod = O.qi_search(J, h, K, iters, phi[r], flips=fl)["productive"]
            m = int(I.unpack_bits(phi[r], n).sum())      # exchanges keep the magnetisation
            want_p += prod * {0: n * (n - 1) // 2, 1: 0, 2: m * (n - m)}[fl]
            want_s += prod * (0 if fl == 2 else n)
        assert (pairs, singles) == (want_p, want_s), name
        ctx.close()


def test_exchange_gaussian_n600_120x64_sampled():
    """120 instances, n = 600, K = 120, R = 64, split-BF16, exchanges; sampled searches."""
    n, K, R, iters, n_inst = 600, 120, 64, 120, 120
    ctx = qis.Context(K=K, R=R, precision="split_bf16", max_n=n, max_instances=n_inst, flips="exchange")
    data = []
    for k in range(n_inst):
        J, h = I.instance("gaussian", n, seed=240, inst=k)
        phi = I.random_states(n, R, seed=241, inst=k)
        ctx.create_instance(J, h)
        ctx.init_states(k, phi)
        data.append((J, h, phi))
    ctx.iterate(iters)
    rng = np.random.default_rng(0)
    for k, r in [(int(rng.integers(n_inst)), int(rng.integers(R))) for _ in range(3)]:
        J, h, phi = data[k]
        same(ctx.search_list(k, r), O.qi_search(J, h, K, iters, phi[r], flips=2), f"inst={k} r={r}")
    ctx.close()
