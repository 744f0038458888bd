"""Parity at the full sizes of the benchmark workloads (Alg. 3 lists and the Alg. 4 merge).

The GPU runs every search of the workload in one context, exactly as the benchmark does; the
oracle re-runs a spread sample of those searches, and the complete Alg. 4 multi-search of a
few instances, in a pool of host processes (spawned, so no process is forked from one that
holds a GPU context). Comparisons:

  * grid inputs (the seeded ensembles; every energy an exact FP64 number): each sampled
    search's kept list equal bit for bit (states, energies, used flags, stamps), the merged list
    equal in states and sources, its rescored energies within 1e-9 relative;
  * unrounded N(0, 1) FP64 inputs (the Gaussian ensemble as drawn, not on any grid): the library
    represents them on its exact grid 2^-q (q capped by the 2^52 bound on every energy sum; the
    instance is flagged as rounded) while the oracle runs on the values as given, so the kept
    states, stamps and used flags must be identical and the energies agree within 1e-9 relative.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

from paper_2010_00180_gb300 import build, inputs as I, qis

pytestmark = pytest.mark.gpu

RTOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    qis.load()


@pytest.fixture(scope="module")
def pool():
    from oracle import oracle as O
    O.build()
    with mp.get_context("spawn").Pool(max(2, min(16, os.cpu_count() or 2))) as p:
        yield p


def _inst(spec, k):
    ens, n, seed, grid = spec
    return I.instance(ens, n, seed=seed, inst=k, grid_bits=grid)


def _states(spec, k, R):
    ens, n, seed, grid = spec
    return I.random_states(n, R, seed=seed + 1000, inst=k)


def _search_job(a):
    spec, k, r, R, K, iters = a
    from oracle import oracle as O
    J, h = _inst(spec, k)
    res = O.qi_search(J, h, K, iters, _states(spec, k, R)[r])
    c = res["count"]
    return k, r, {x: res[x][:c] for x in ("bits", "E", "used", "stamp")}


def _multi_job(a):
    spec, k, R, K, iters = a
    from oracle import oracle as O
    J, h = _inst(spec, k)
    return k, O.qi_multi_search(J, h, K, iters, _states(spec, k, R))


def run_gpu(specs, R, K, iters, precision):
    """One context with every instance of `specs` (list of (spec, k)), iterated `iters` times."""
    ns = [s[0][1] for s in specs]
    ctx = qis.Context(K=K, R=R, precision=precision, max_n=max(ns), max_instances=len(specs))
    pairs = [_inst(spec, k) for spec, k in specs]
    ids = ctx.create_instances(pairs)
    for iid, (spec, k) in zip(ids, specs):
        ctx.init_states(iid, _states(spec, k, R))
    ctx.iterate(iters)
    ctx.synchronize()
    return ctx


def check(ctx, pool, specs, R, K, iters, sample, merged, exact_E=True):
    """sample: [(index in specs, r)]; merged: [index in specs] compared after Alg. 4."""
    jobs = [(specs[i][0], specs[i][1], r, R, K, iters) for i, r in sample]
    mjobs = [(specs[i][0], specs[i][1], R, K, iters) for i in merged]
    m_async = pool.map_async(_multi_job, mjobs)
    where = {(specs[i][0], specs[i][1]): i for i in range(len(specs))}
    for (k, r, ref), (i, _) in zip(pool.map(_search_job, jobs), sample):
        got = ctx.search_list(i, r)
        what = f"instance {i} (n={specs[i][0][1]}) search {r}"
        assert got["count"] == len(ref["E"]), what
        assert np.array_equal(got["bits"], ref["bits"]), what
        assert np.array_equal(got["used"], ref["used"]), what
        assert np.array_equal(got["stamp"], ref["stamp"]), what
        if exact_E:
            assert np.array_equal(got["E"], ref["E"]), what
        else:
            np.testing.assert_allclose(got["E"], ref["E"], rtol=RTOL, atol=0, err_msg=what)
    for i, ref in zip(merged, [x[1] for x in m_async.get()]):
        got = ctx.topk_states(i, K + 1)
        what = f"merged list of instance {i}"
        assert got["count"] == ref["count"], what
        assert np.array_equal(got["bits"], ref["bits"]), what
        assert np.array_equal(got["src"], ref["src"]), what
        np.testing.assert_allclose(got["E"], ref["E"], rtol=RTOL, atol=0, err_msg=what)


def spread(n_inst, R, count, seed):
    """`count` (instance, search) pairs spread over every instance: instance floor(t n_inst /
    count) with a seeded random search."""
    rng = np.random.default_rng(seed)
    return [((t * n_inst) // count, int(rng.integers(R))) for t in range(count)]


def test_gaussian_n600_120x64_split_full_size(pool):
    """120 instances, n = 600, K = 120, R = 64, I = 120 (the benchmark's default workload):
    64 searches over all 120 instances, and the Alg. 4 merged lists of three instances."""
    spec = ("gaussian", 600, 3, I.GRID_BITS)
    specs = [(spec, k) for k in range(120)]
    ctx = run_gpu(specs, 64, 120, 120, "split_bf16")
    check(ctx, pool, specs, 64, 120, 120, spread(120, 64, 64, 1), merged=[0, 57, 119])
    ctx.close()


def test_pm1_n1024_64x128_full_size(pool):
    """64 instances, n = 1024, J = +-1, h in {-1, 0, 1}, K = 120, R = 128, I = 120: 32 searches
    over all 64 instances (bit-exact), and the Alg. 4 merged lists of three instances."""
    spec = ("pm1", 1024, 4, I.GRID_BITS)
    specs = [(spec, k) for k in range(64)]
    ctx = run_gpu(specs, 128, 120, 120, "pm1_fp8")
    check(ctx, pool, specs, 128, 120, 120, spread(64, 128, 32, 2), merged=[0, 31, 63])
    ctx.close()


def test_mixed_sizes_200_350_500_700_full_size(pool):
    """The mixed batch n in {200, 350, 500, 700} at the +-J workload's K = 120, R = 128, I = 120
    in one context: 8 searches of each instance, and the merged lists of n = 200 and n = 700."""
    specs = [(("pm1", n, 44, I.GRID_BITS), k) for k, n in enumerate([200, 350, 500, 700])]
    ctx = run_gpu(specs, 128, 120, 120, "pm1_fp8")
    rng = np.random.default_rng(3)
    sample = [(i, int(r)) for i in range(4) for r in rng.choice(128, 8, replace=False)]
    check(ctx, pool, specs, 128, 120, 120, sample, merged=[0, 3])
    ctx.close()


def test_unrounded_fp64_gaussian_n600_120x64(pool):
    """The default workload's size with N(0, 1) couplings and fields as drawn in FP64 (no grid):
    the library flags every instance as rounded onto its exact grid; 32 searches over all 120
    instances and the merged list of one keep the oracle's states, stamps and used flags, with
    energies within 1e-9 relative."""
    spec = ("gaussian", 600, 5, None)
    specs = [(spec, k) for k in range(120)]
    ctx = run_gpu(specs, 64, 120, 120, "split_bf16")
    q, _, rounded = ctx.instance_info(0)
    assert rounded and q >= 30
    J, _ = _inst(spec, 0)
    assert np.any(J * 2.0 ** 40 != np.rint(J * 2.0 ** 40))      # really off any fine grid
    check(ctx, pool, specs, 64, 120, 120, spread(120, 64, 32, 4), merged=[60], exact_E=False)
    ctx.close()
