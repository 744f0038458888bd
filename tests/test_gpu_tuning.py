"""Launch shapes and the autotuner: no setting may change a result (the scan's chunking and
search grouping and the GEMM tile only move work between blocks)."""
import numpy as np
import pytest

from paper_2010_00180_gb300 import build, inputs as I, qis

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    qis.load()


def make(ens, prec, ns, K=20, R=12):
    ctx = qis.Context(K=K, R=R, precision=prec, max_n=max(ns), max_instances=len(ns))
    for k, n in enumerate(ns):
        J, h = I.instance(ens, n, seed=40, inst=k)
        ctx.create_instance(J, h)
        ctx.init_states(k, I.random_states(n, R, seed=41, inst=k))
    return ctx


def lists(ctx, n_inst, R):
    return [[ctx.search_list(k, r) for r in range(R)] for k in range(n_inst)]


@pytest.mark.parametrize("ens,prec", [("gaussian", "split_bf16"), ("pm1", "pm1_fp8"), ("gaussian", "fp64")])
def test_results_do_not_depend_on_launch_shapes(ens, prec):
    ns, R, iters = [100, 257, 64], 12, 12
    ctx = make(ens, prec, ns, R=R)
    ctx.iterate(iters)
    want = lists(ctx, len(ns), R)
    settings = [(4, 0, 0), (2, 3, 16), (6, 4, 32), (1, 12, 0), (8, 5, 48), (3, 1, 0)]
    for nc, rg, nt in settings:
        if prec == "fp64":
            nt = 0
        ctx.set_tuning(nc, rg, nt)
        got = ctx.tuning()
        assert got["scan_chunk_nc"] == nc and got["scan_search_group"] == (rg or R)
        ctx.reset()
        ctx.iterate(iters)
        have = lists(ctx, len(ns), R)
        for k in range(len(ns)):
            for r in range(R):
                for key in ("bits", "E", "stamp", "used"):
                    assert np.array_equal(have[k][r][key], want[k][r][key]), (nc, rg, nt, k, r, key)
    ctx.close()


def test_autotune_resets_and_keeps_results():
    ns, R = [300, 300], 16
    ctx = make("gaussian", "split_bf16", ns, R=R)
    ctx.iterate(10)
    want = lists(ctx, len(ns), R)
    best = ctx.autotune(4)
    assert 1 <= best["scan_chunk_nc"] <= 8 and 1 <= best["scan_search_group"] <= R and best["ms"] > 0
    for k, n in enumerate(ns):
        init = I.random_states(n, R, seed=41, inst=k)
        for r in range(R):
            lst = ctx.search_list(k, r)
            assert lst["count"] == 1 and np.array_equal(lst["bits"][0], init[r])
    ctx.iterate(10)
    have = lists(ctx, len(ns), R)
    for k in range(len(ns)):
        for r in range(R):
            assert np.array_equal(have[k][r]["bits"], want[k][r]["bits"])
            assert np.array_equal(have[k][r]["E"], want[k][r]["E"])
    ctx.close()


def test_invalid_tuning_is_rejected():
    ctx = make("gaussian", "split_bf16", [80], R=8)
    before = ctx.tuning()
    for bad in [(0, 0, 0), (9, 0, 0), (8, 9, 0), (8, -1, 0), (8, 0, 24), (8, 0, 512)]:
        with pytest.raises(qis.QISError) as e:
            ctx.set_tuning(*bad)
        assert e.value.name == "INVALID_ARG"
        assert ctx.tuning() == before
    ctx.close()
