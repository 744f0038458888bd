"""The output-sensitive pair scan (live rows, columns ordered by a bucket of a_j, each live
row's bucket prefix) against the dense register-tile scan (QIS_DENSE_SCAN=1): both test every
pair that can pass with the same arithmetic, so every search must come out identical, and
equal to the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2010_00180_gb300 import build, inputs as I, qis

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    qis.load()


def run(prec, ens, flips, ns, K, R, iters, seed):
    ctx = qis.Context(K=K, R=R, precision=prec, max_n=max(ns), max_instances=len(ns), flips=flips)
    data = [I.instance(ens, n, seed=seed, inst=k) for k, n in enumerate(ns)]
    phis = [I.random_states(n, R, seed=seed + 1, inst=k) for k, n in enumerate(ns)]
    ctx.create_instances(data)
    for k in range(len(ns)):
        ctx.init_states(k, phis[k])
    ctx.iterate(iters)
    lists = [[ctx.search_list(k, r) for r in range(R)] for k in range(len(ns))]
    ctx.close()
    return data, phis, lists


@pytest.mark.parametrize("prec,ens,flips", [("split_bf16", "gaussian", "single_pair"),
                                            ("pm1_fp8", "pm1", "single_pair"),
                                            ("split_bf16", "uniform", "exchange"),
                                            ("pm1_fp8", "pm1", "exchange")])
def test_sparse_equals_dense(prec, ens, flips, monkeypatch):
    ns, K, R, iters = [300, 171, 64], 40, 8, 30
    _, _, sparse = run(prec, ens, flips, ns, K, R, iters, 600)
    monkeypatch.setenv("QIS_DENSE_SCAN", "1")
    data, phis, dense = run(prec, ens, flips, ns, K, R, iters, 600)
    for k in range(len(ns)):
        for r in range(R):
            for key in ("count", "bits", "E", "stamp", "used"):
                assert np.array_equal(sparse[k][r][key], dense[k][r][key]), (k, r, key)
    J, h = data[0]
    fl = {"single_pair": 0, "exchange": 2}[flips]
    for r in range(2):
        ref = O.qi_search(J, h, K, iters, phis[0][r], flips=fl)
        assert np.array_equal(sparse[0][r]["bits"], ref["bits"][: ref["count"]])


@pytest.mark.parametrize("flips", ["single_pair", "exchange"])
def test_sparse_equals_dense_several_staging_passes(flips, monkeypatch):
    """n = 1500: a block stages its sites in three passes of 640."""
    ns, K, R, iters = [1500, 700], 60, 4, 12
    _, _, sparse = run("split_bf16", "gaussian", flips, ns, K, R, iters, 610)
    monkeypatch.setenv("QIS_DENSE_SCAN", "1")
    _, _, dense = run("split_bf16", "gaussian", flips, ns, K, R, iters, 610)
    for k in range(len(ns)):
        for r in range(R):
            for key in ("count", "bits", "E", "stamp", "used"):
                assert np.array_equal(sparse[k][r][key], dense[k][r][key]), (k, r, key)
