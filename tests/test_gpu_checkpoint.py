"""Checkpoint/resume, list import and the sharded layout on the GPU.

A resumed search must continue exactly as the uninterrupted one (same lists, stamps, used
flags), and lists computed in separate contexts (the processes of a sharded run, emulated
here one after another on one GPU) must merge to the single-context Alg. 4 result."""
import os

import numpy as np
import pytest

from paper_2010_00180_gb300 import build, inputs as I, qis
from paper_2010_00180_gb300 import sharding as S

pytestmark = pytest.mark.gpu

MODES = [("gaussian", "split_bf16"), ("gaussian", "fp64"), ("pm1", "pm1_fp8")]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    qis.load()


def make_ctx(ens, prec, ns, K=20, R=4, seed=30):
    ctx = qis.Context(K=K, R=R, precision=prec, max_n=max(ns), max_instances=len(ns))
    for k, n in enumerate(ns):
        J, h = I.instance(ens, n, seed=seed, inst=k)
        ctx.create_instance(J, h)
        ctx.init_states(k, I.random_states(n, R, seed=seed + 1, inst=k))
    return ctx


def snapshot(ctx, n_inst, R):
    return [[ctx.search_list(k, r) for r in range(R)] for k in range(n_inst)]


def same_lists(a, b):
    for la, lb in zip(a, b):
        for x, y in zip(la, lb):
            assert x["count"] == y["count"]
            for key in ("bits", "E", "used", "stamp"):
                assert np.array_equal(x[key], y[key]), key


@pytest.mark.parametrize("ens,prec", MODES)
def test_save_load_resume_is_exact(tmp_path, ens, prec):
    ns, R = [100, 67], 4
    path = str(tmp_path / "ck.bin")
    a = make_ctx(ens, prec, ns, R=R)
    a.iterate(7)
    a.save(path)
    a.iterate(8)
    want = snapshot(a, len(ns), R)
    top_a = [a.topk_states(k, 21) for k in range(len(ns))]
    a.close()
    b = qis.Context(K=20, R=R, precision=prec, max_n=128, max_instances=4)
    b.load(path)
    assert [b.n[k] for k in range(len(ns))] == ns
    b.iterate(8)
    same_lists(want, snapshot(b, len(ns), R))
    for k in range(len(ns)):
        t = b.topk_states(k, 21)
        assert np.array_equal(t["bits"], top_a[k]["bits"]) and np.array_equal(t["E"], top_a[k]["E"])
    # reset after load goes back to the stored initial states
    b.reset()
    for k, n in enumerate(ns):
        for r in range(R):
            assert np.array_equal(b.search_list(k, r)["bits"][0], I.random_states(n, R, seed=31, inst=k)[r])
    b.close()


def test_load_rejects_bad_files(tmp_path):
    path = str(tmp_path / "ck.bin")
    a = make_ctx("gaussian", "split_bf16", [40])
    a.iterate(3)
    a.save(path)
    a.close()
    raw = open(path, "rb").read()
    bad = bytearray(raw)
    bad[len(raw) // 2] ^= 0x10
    open(str(tmp_path / "flip.bin"), "wb").write(bytes(bad))
    open(str(tmp_path / "short.bin"), "wb").write(raw[:-9])
    b = qis.Context(K=20, R=4, precision="split_bf16", max_n=64)
    for name in ("flip.bin", "short.bin", "missing.bin"):
        with pytest.raises(qis.QISError) as e:
            b.load(str(tmp_path / name))
        assert e.value.name == "INVALID_ARG"
    c = qis.Context(K=21, R=4, precision="split_bf16", max_n=64)     # K differs
    with pytest.raises(qis.QISError):
        c.load(path)
    c.close()
    b.load(path)                                   # the context is still usable
    with pytest.raises(qis.QISError) as e:
        b.load(path)                               # it now holds instances
    assert e.value.name == "STATE"
    b.iterate(2)
    b.close()


def test_load_failing_part_way_leaves_no_instances(tmp_path):
    """A checkpoint whose second instance does not fit the context (n = 80 > max_n = 60) fails
    after the first instance was created: the load removes it again, so a retry with a good
    file succeeds in the same context and continues the saved searches exactly."""
    big, good = str(tmp_path / "two.bin"), str(tmp_path / "one.bin")
    a = make_ctx("gaussian", "split_bf16", [40, 80])
    a.iterate(3)
    a.save(big)
    a.close()
    a = make_ctx("gaussian", "split_bf16", [40])
    a.iterate(3)
    a.save(good)
    a.iterate(4)
    want = snapshot(a, 1, 4)
    a.close()
    b = qis.Context(K=20, R=4, precision="split_bf16", max_n=60, max_instances=2)
    with pytest.raises(qis.QISError) as e:
        b.load(big)
    assert e.value.name == "INVALID_ARG" and "max_n" in str(e.value)
    assert b.lib.qis_instance_n(b.h, 0, None) != 0          # no instance left behind
    b.load(good)
    b.iterate(4)
    same_lists(want, snapshot(b, 1, 4))
    b.close()


def test_set_search_list_roundtrip_and_checks():
    a = make_ctx("gaussian", "split_bf16", [90], R=2)
    a.iterate(5)
    src = a.search_list(0, 1)
    b = make_ctx("gaussian", "split_bf16", [90], R=2)
    b.set_search_list(0, 0, src["bits"], src["E"], src["used"], src["stamp"], t=5)
    got = b.search_list(0, 0)
    for key in ("bits", "E", "used", "stamp"):
        assert np.array_equal(got[key], src[key]), key
    bits, E = src["bits"], src["E"]
    bad_cases = [
        (bits[:0], E[:0]),                                        # empty
        (bits[[1, 0]], E[[1, 0]]) if E[1] > E[0] else None,      # energies not ascending
        (bits[[0, 0]], E[[0, 0]]),                                # duplicate state
        (np.concatenate([bits, bits[:1]]), np.concatenate([E, [E[-1] + 1]])) if len(E) == 21 else None,
    ]
    hi = bits[:1].copy()
    hi[0, -1] |= np.uint64(1) << np.uint64(63)                    # bit above n = 90
    bad_cases.append((hi, E[:1]))
    for case in bad_cases:
        if case is None:
            continue
        with pytest.raises(qis.QISError) as e:
            b.set_search_list(0, 1, case[0], case[1])
        assert e.value.name == "INVALID_ARG"
    a.close()
    b.close()


@pytest.mark.parametrize("n_inst,R,world", [(1, 8, 2), (3, 4, 2), (2, 6, 4)])
def test_sharded_run_equals_single_context(n_inst, R, world):
    """Every process of a world-size run, one after another on this GPU (they never wait on
    one another), then the owners' merges: identical to one context running everything."""
    n, K, iters = 72, 16, 12
    instances = [I.instance("gaussian", n, seed=90, inst=k) for k in range(n_inst)]
    states = [I.random_states(n, R, seed=91, inst=k) for k in range(n_inst)]
    shards = S.plan(n_inst, R, world)
    lists, tops = {}, {}
    for rank in range(world):
        ctx, ids, loc = S.run_local(instances, states, shards[rank], K, iters)
        lists.update(loc)
        if ctx is not None:
            for inst, iid in ids.items():
                if inst not in S.split_instances(shards):
                    tops[inst] = ctx.topk_states(iid, K + 1)
            ctx.close()
    split = S.split_instances(shards)
    gathered = {i: [lists[(i, r)] for r in range(R)] for i in split}
    tops.update(S.merge_gathered(instances, states, gathered, K))
    ref = qis.Context(K=K, R=R, precision="split_bf16", max_n=n, max_instances=n_inst)
    for k, (J, h) in enumerate(instances):
        ref.create_instance(J, h)
        ref.init_states(k, states[k])
    ref.iterate(iters)
    for k in range(n_inst):
        want = ref.topk_states(k, K + 1)
        for key in ("bits", "E", "src"):
            assert np.array_equal(tops[k][key], want[key]), (k, key)
    ref.close()
