"""Batched instance creation (one validation read-back for many instances) and the exact
integer rescoring of grid instances: the same instances, descriptors and searches as one call
per instance; an invalid member adds nothing; energies equal numpy's FP64 ones."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2010_00180_gb300 import build, inputs as I, qis

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    qis.load()


def energy_np(J, h, S):
    return np.einsum("mi,ij,mj->m", S, np.triu(J, 1), S) + S @ h


@pytest.mark.parametrize("prec,ens", [("split_bf16", "gaussian"), ("pm1_fp8", "pm1"), ("fp64", "gaussian")])
def test_batch_equals_one_by_one(prec, ens):
    ns, K, R, iters = [90, 150, 64, 121], 24, 6, 20
    data = [I.instance(ens, n, seed=400, inst=k) for k, n in enumerate(ns)]
    phis = [I.random_states(n, R, seed=401, inst=k) for k, n in enumerate(ns)]
    out = []
    for batched in (True, False):
        ctx = qis.Context(K=K, R=R, precision=prec, max_n=max(ns), max_instances=len(ns))
        if batched:
            ids = ctx.create_instances(data)
        else:
            ids = [ctx.create_instance(J, h) for J, h in data]
        assert ids == list(range(len(ns)))
        infos = [ctx.instance_info(k) for k in ids]
        for k in ids:
            ctx.init_states(k, phis[k])
        ctx.iterate(iters)
        lists = [[ctx.search_list(k, r) for r in range(R)] for k in ids]
        tops = [ctx.topk_states(k, K + 1) for k in ids]
        out.append((infos, lists, tops))
        ctx.close()
    assert out[0][0] == out[1][0]
    for k in range(len(ns)):
        for r in range(R):
            for key in ("count", "bits", "E", "stamp", "used"):
                assert np.array_equal(out[0][1][k][r][key], out[1][1][k][r][key]), (k, r, key)
        for key in ("count", "bits", "E", "src"):
            assert np.array_equal(out[0][2][k][key], out[1][2][k][key]), (k, key)
    # and the searches are the oracle's
    J, h = data[1]
    for r in range(R):
        ref = O.qi_search(J, h, K, iters, phis[1][r])
        got = out[0][1][1][r]
        assert np.array_equal(got["bits"], ref["bits"][: ref["count"]])


def _pinned(a):
    """A page-locked host copy of a (numpy view of a pinned torch tensor)."""
    import torch
    t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
    out = t.numpy()
    out[...] = a
    return out, t


@pytest.mark.parametrize("prec,ens", [("split_bf16", "gaussian"), ("pm1_fp8", "pm1")])
def test_page_locked_inputs_equal_pageable(prec, ens):
    """A page-locked J is read by the layout kernel directly (no staging copy): a batch mixing
    page-locked and pageable couplings gives the same instances and searches as pageable ones;
    an invalid page-locked J is rejected the same way."""
    ns, K, R, iters = [90, 150, 64], 16, 4, 12
    data = [I.instance(ens, n, seed=405, inst=k) for k, n in enumerate(ns)]
    phis = [I.random_states(n, R, seed=406, inst=k) for k, n in enumerate(ns)]
    keep = []
    mixed = []
    for k, (J, h) in enumerate(data):
        if k != 1:
            Jp, t = _pinned(J)
            keep.append(t)
            mixed.append((Jp, h))
        else:
            mixed.append((J, h))
    out = []
    for batch in (data, mixed):
        ctx = qis.Context(K=K, R=R, precision=prec, max_n=max(ns), max_instances=len(ns))
        ids = ctx.create_instances(batch)
        infos = [ctx.instance_info(k) for k in ids]
        for k in ids:
            ctx.init_states(k, phis[k])
        ctx.iterate(iters)
        lists = [[ctx.search_list(k, r) for r in range(R)] for k in ids]
        out.append((infos, lists, ctx.topk_states_all(K + 1)))
        ctx.close()
    assert out[0][0] == out[1][0]
    for k in range(len(ns)):
        for r in range(R):
            for key in ("count", "bits", "E", "stamp"):
                assert np.array_equal(out[0][1][k][r][key], out[1][1][k][r][key]), (k, r, key)
        for key in ("count", "bits", "E", "src"):
            assert np.array_equal(out[0][2][k][key], out[1][2][k][key]), (k, key)
    J, h = data[0]
    Jbad, t = _pinned(J)
    Jbad[2, 7] += 1.0   # no longer symmetric
    ctx = qis.Context(K=K, R=R, precision=prec, max_n=max(ns), max_instances=2)
    with pytest.raises(qis.QISError) as e:
        ctx.create_instances([(Jbad, h)])
    assert e.value.name == "INVALID_ARG"
    ctx.close()


def test_invalid_member_adds_nothing():
    ctx = qis.Context(K=8, R=2, precision="split_bf16", max_n=40, max_instances=4)
    good = I.instance("gaussian", 30, seed=410)
    J, h = I.instance("gaussian", 30, seed=411)
    J = J.copy()
    J[3, 5] += 1.0   # no longer symmetric
    with pytest.raises(qis.QISError) as e:
        ctx.create_instances([good, (J, h), good])
    assert e.value.name == "INVALID_ARG"
    assert ctx.create_instances([good]) == [0]   # nothing of the failed batch was added
    ctx.close()


@pytest.mark.parametrize("ens", ["gaussian", "uniform", "pm1"])
def test_exact_rescoring_equals_fp64_energies(ens):
    """Grid instances are rescored in exact integers; the result is the FP64 energy (every
    partial sum of grid numbers is exact), for any summation order."""
    n = 200
    prec = "pm1_fp8" if ens == "pm1" else "split_bf16"
    J, h = I.instance(ens, n, seed=420)
    ctx = qis.Context(K=8, R=2, precision=prec, max_n=n, max_instances=1)
    ctx.create_instance(J, h)
    assert ctx.instance_info(0)[2] == 0   # on its grid: not rounded
    bits = I.random_states(n, 300, seed=421)
    E = ctx.energies(0, bits)
    S = 1.0 - 2.0 * I.unpack_bits(bits, n).astype(np.float64)
    assert np.array_equal(E, energy_np(J, h, S))
    ctx.close()


def test_rounded_instance_keeps_fp64_rescoring():
    """Couplings off any usable grid are rounded for the search, but energies are still the
    FP64 energies of the given couplings."""
    n = 60
    rng = np.random.default_rng(430)
    J = np.triu(rng.standard_normal((n, n)), 1)
    J = J + J.T
    h = rng.standard_normal(n)
    ctx = qis.Context(K=8, R=2, precision="split_bf16", max_n=n, max_instances=1)
    ctx.create_instance(J, h)
    assert ctx.instance_info(0)[2] == 1
    bits = I.random_states(n, 50, seed=431)
    E = ctx.energies(0, bits)
    S = 1.0 - 2.0 * I.unpack_bits(bits, n).astype(np.float64)
    np.testing.assert_allclose(E, energy_np(J, h, S), rtol=1e-12, atol=1e-12)
    ctx.close()


@pytest.mark.parametrize("prec,ens", [("split_bf16", "gaussian"), ("fp64", "gaussian"), ("pm1_fp8", "pm1")])
def test_topk_all_equals_per_instance(prec, ens):
    ns, K, R, iters = [70, 130, 45], 20, 5, 15
    ctx = qis.Context(K=K, R=R, precision=prec, max_n=max(ns), max_instances=len(ns))
    data = [I.instance(ens, n, seed=440, inst=k) for k, n in enumerate(ns)]
    ctx.create_instances(data)
    for k, n in enumerate(ns):
        ctx.init_states(k, I.random_states(n, R, seed=441, inst=k))
    ctx.iterate(iters)
    for kk in (K + 1, 7):
        every = ctx.topk_states_all(kk)
        for k in range(len(ns)):
            one = ctx.topk_states(k, kk)
            assert every[k]["count"] == one["count"]
            for key in ("bits", "E", "src"):
                assert np.array_equal(every[k][key], one[key]), (kk, k, key)
    ctx.close()


@pytest.mark.parametrize("smem_cand", ["32", "512"])
def test_merge_overflow_buffer_pm1_ties(smem_cand, monkeypatch):
    """+-J couplings with h = 0 tie many candidates at the threshold, so a search keeps more
    survivors than the merge holds in shared memory (32 slots forced here; 512 is the default):
    the overflow buffer in global memory must give the same lists as the oracle."""
    monkeypatch.setenv("QIS_MERGE_SMEM_CAND", smem_cand)
    n, K, R, iters = 300, 120, 3, 6
    J, _ = I.instance("pm1", n, seed=450)
    h = np.zeros(n)
    phi = I.random_states(n, R, seed=451)
    ctx = qis.Context(K=K, R=R, precision="pm1_fp8", max_n=n, max_instances=1, survivor_cap=16384)
    ctx.create_instance(J, h)
    ctx.init_states(0, phi)
    for t in range(1, iters + 1):
        ctx.iterate(1)
        for r in range(R):
            ref = O.qi_search(J, h, K, t, phi[r])
            got = ctx.search_list(0, r)
            c = ref["count"]
            assert got["count"] == c
            for key in ("bits", "E", "used", "stamp"):
                assert np.array_equal(got[key], ref[key][:c]), (t, r, key)
    ctx.close()
