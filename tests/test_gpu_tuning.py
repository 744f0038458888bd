"""Launch shapes and the autotuner: no setting may change a result (the pair filter's form,
the dense scan's chunking and search grouping and the GEMM tile only move work between
blocks)."""
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
    # the dense form (2) with its chunk widths and search groups, the output-sensitive form (1)
    settings = [(4, 0, 0, 2), (2, 3, 16, 2), (6, 4, 32, 1), (1, 12, 0, 2), (8, 5, 48, 1), (3, 1, 0, 2),
                (8, 0, 0, 0)]
    for nc, rg, nt, ps in settings:
        if prec == "fp64":
            nt, ps = 0, (0 if ps == 1 else ps)
        ctx.set_tuning(nc, rg, nt, ps)
        got = ctx.tuning()
        assert got["scan_chunk_nc"] == nc and got["scan_search_group"] == (rg or R)
        assert got["pair_scan"] == (2 if prec == "fp64" else (ps or 1))
        ctx.reset()
        ctx.iterate(iters)
        have = lists(ctx, len(ns), R)
        for k in range(len(ns)):
            for r in range(R):
                for key in ("bits", "E", "stamp", "used"):
                    assert np.array_equal(have[k][r][key], want[k][r][key]), (nc, rg, nt, ps, k, r, key)
    ctx.close()


def test_autotune_resets_and_keeps_results():
    ns, R = [300, 300], 16
    ctx = make("gaussian", "split_bf16", ns, R=R)
    ctx.iterate(10)
    want = lists(ctx, len(ns), R)
    best = ctx.autotune(4)
    assert 1 <= best["scan_chunk_nc"] <= 8 and 1 <= best["scan_search_group"] <= R and best["ms"] > 0
    assert best["pair_scan"] in (1, 2) and ctx.tuning()["pair_scan"] == best["pair_scan"]
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
    for bad in [(0, 0, 0), (9, 0, 0), (8, 9, 0), (8, -1, 0), (8, 0, 24), (8, 0, 512), (8, 0, 0, 4), (8, 0, 0, -1)]:
        with pytest.raises(qis.QISError) as e:
            ctx.set_tuning(*bad)
        assert e.value.name == "INVALID_ARG"
        assert ctx.tuning() == before
    ctx.close()


def test_output_sensitive_scan_refused_where_it_cannot_run():
    """pair_scan 1 needs a split mode and a padded size of at most 4096."""
    for prec, n in (("fp64", 50), ("split_bf16", 4200)):
        ctx = qis.Context(K=8, R=2, precision=prec, max_n=n, max_instances=1)
        assert ctx.tuning()["pair_scan"] == 2
        with pytest.raises(qis.QISError) as e:
            ctx.set_tuning(8, 0, 0, 1)
        assert e.value.name == "INVALID_ARG"
        assert ctx.tuning()["pair_scan"] == 2
        ctx.close()
