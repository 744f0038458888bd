"""Local fields by update (fq of a child = fq of its generating parent minus the flipped sites'
coupling columns) against the field GEMM and the oracle: identical lists with the update on
and off, a two-slot field ring that forces the GEMM fallback for older generators, imported
lists, and the FP64 mode's refusal."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2010_00180_gb300 import build, inputs as I, qis

pytestmark = pytest.mark.gpu

MODES = [("split_bf16", "gaussian"), ("pm1_fp8", "pm1")]
FLIPS = ["single_pair", "single", "exchange"]
FLIP_CODE = {"single_pair": 0, "single": 1, "exchange": 2}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    qis.load()


def make(prec, ens, ns, K, R, flips="single_pair", seed=300):
    ctx = qis.Context(K=K, R=R, precision=prec, max_n=max(ns), max_instances=len(ns), flips=flips)
    data = []
    for k, n in enumerate(ns):
        J, h = I.instance(ens, n, seed=seed, inst=k)
        phi = I.random_states(n, R, seed=seed + 1, inst=k)
        ctx.create_instance(J, h)
        ctx.init_states(k, phi)
        data.append((J, h, phi))
    return ctx, data


def lists(ctx, n_inst, R):
    return [[ctx.search_list(k, r) for r in range(R)] for k in range(n_inst)]


def same(g, o, what=""):
    c = o["count"]
    assert g["count"] == c, what
    for key in ("bits", "E", "used", "stamp"):
        assert np.array_equal(g[key], o[key][:c]), (what, key)


@pytest.mark.parametrize("flips", FLIPS)
@pytest.mark.parametrize("prec,ens", MODES)
def test_update_equals_gemm(prec, ens, flips):
    ns, K, R, iters = [150, 97, 64], 30, 20, 40
    got = []
    for on in (True, False):
        ctx, _ = make(prec, ens, ns, K, R, flips)
        ctx.set_incremental_fields(on)
        ctx.iterate(iters)
        got.append(lists(ctx, len(ns), R))
        ctx.close()
    for k in range(len(ns)):
        for r in range(R):
            for key in ("count", "bits", "E", "stamp", "used"):
                assert np.array_equal(got[0][k][r][key], got[1][k][r][key]), (k, r, key)


@pytest.mark.parametrize("prec,ens", MODES)
def test_two_slot_ring_falls_back_to_the_gemm(prec, ens, monkeypatch):
    """Past the descent a parent's generator is often more than two iterations back: those
    parents take the GEMM's fields, the others the update; every iteration equals the oracle."""
    monkeypatch.setenv("QIS_FIELD_RING", "2")
    n, K, R, iters = 48, 24, 6, 90
    ctx, data = make(prec, ens, [n], K, R, seed=310)
    J, h, phi = data[0]
    for t in range(1, iters + 1):
        ctx.iterate(1)
        if t % 10 == 0 or t < 6:
            for r in range(R):
                same(ctx.search_list(0, r), O.qi_search(J, h, K, t, phi[r]), f"t={t} r={r}")
    ctx.close()


def test_imported_list_gets_full_fields():
    """Entries of an imported list have no generator fields in the ring."""
    n, K, R = 80, 20, 4
    ctx, data = make("split_bf16", "gaussian", [n], K, R, seed=320)
    J, h, phi = data[0]
    ctx.iterate(12)
    saved = [ctx.search_list(0, r) for r in range(R)]
    ctx2, _ = make("split_bf16", "gaussian", [n], K, R, seed=320)
    for r in range(R):
        s = saved[r]
        ctx2.set_search_list(0, r, s["bits"], s["E"], s["used"], s["stamp"], 12)
    ctx.iterate(15)
    ctx2.iterate(15)
    for r in range(R):
        a, b = ctx.search_list(0, r), ctx2.search_list(0, r)
        for key in ("count", "bits", "E", "stamp", "used"):
            assert np.array_equal(a[key], b[key]), (r, key)
        same(a, O.qi_search(J, h, K, 27, phi[r]), f"r={r}")
    ctx.close()
    ctx2.close()


def test_fp64_mode_refuses_the_update():
    ctx, _ = make("fp64", "gaussian", [40], 8, 2)
    with pytest.raises(qis.QISError) as e:
        ctx.set_incremental_fields(True)
    assert e.value.name == "INVALID_ARG"
    ctx.set_incremental_fields(False)
    ctx.close()
