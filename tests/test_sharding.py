"""Multi-process layout (CPU, gloo): the shard plan covers every search once, and the lists
gathered to an instance's owner give the single-process Alg. 4 result."""
import os
import socket
import sys

import numpy as np
import pytest

from paper_2010_00180_gb300 import inputs as I
from paper_2010_00180_gb300 import sharding as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("n_inst,R,world", [(120, 64, 1), (120, 64, 8), (7, 5, 3), (1, 8, 2), (1, 3, 4),
                                            (2, 6, 5), (3, 1, 8), (0, 4, 2)])
def test_plan_covers_every_search_once(n_inst, R, world):
    shards = S.plan(n_inst, R, world)
    assert len(shards) == world
    seen = {}
    for k, mine in enumerate(shards):
        assert len({s.r1 - s.r0 for s in mine}) <= 1        # one context per process
        for s in mine:
            assert 0 <= s.r0 < s.r1 <= R
            for r in range(s.r0, s.r1):
                assert (s.instance, r) not in seen
                seen[(s.instance, r)] = k
    assert set(seen) == {(i, r) for i in range(n_inst) for r in range(R)}
    for i in range(n_inst):
        assert seen[(i, 0)] == S.owner(shards, i)
    if n_inst >= world:
        assert not S.split_instances(shards)                 # no exchange at all
        sizes = [len(m) for m in shards]
        assert max(sizes) - min(sizes) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, cfg, q):
    try:
        sys.path.insert(0, ROOT)
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        import torch.distributed as dist
        from oracle import oracle as O
        from paper_2010_00180_gb300 import inputs as I
        from paper_2010_00180_gb300 import sharding as S
        dist.init_process_group("gloo", rank=rank, world_size=world)
        n_inst, n, R, K, iters = cfg
        inst = [I.instance("gaussian", n, seed=70, inst=k) for k in range(n_inst)]
        phi = [I.random_states(n, R, seed=71, inst=k) for k in range(n_inst)]
        shards = S.plan(n_inst, R, world)
        local = {}
        for s in shards[rank]:                      # this rank's searches (oracle stands in for the GPU)
            J, h = inst[s.instance]
            for r in range(s.r0, s.r1):
                res = O.qi_search(J, h, K, iters, phi[s.instance][r])
                local[(s.instance, r)] = (res["bits"][: res["count"]], res["E"][: res["count"]])
        got = S.gather_lists(local, shards, rank)
        dist.destroy_process_group()
        q.put((rank, {i: [(b.tolist(), e.tolist()) for b, e in lists] for i, lists in got.items()}, None))
    except Exception as e:  # report instead of hanging the parent
        q.put((rank, None, repr(e)))


@pytest.mark.parametrize("n_inst,R", [(1, 6), (3, 4)])
def test_gather_to_owner_gives_single_process_merge(n_inst, R):
    import multiprocessing as mp
    from oracle import oracle as O
    world, n, K, iters = 2, 14, 10, 10
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(k, world, port, (n_inst, n, R, K, iters), q)) for k in range(world)]
    for p in ps:
        p.start()
    out = {}
    for _ in range(world):
        rank, got, err = q.get(timeout=240)
        assert err is None, err
        out[rank] = got
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    shards = S.plan(n_inst, R, world)
    split = S.split_instances(shards)
    assert split == (set(range(n_inst)) if n_inst < world else set())
    for i in split:
        own = S.owner(shards, i)
        lists = out[own][i]
        assert len(lists) == R
        for k in range(world):
            if k != own:
                assert i not in out[k]
        # Alg. 4 from the gathered lists: union in search order, first occurrence, (E, r, pos)
        seen = {}
        for r, (bits, E) in enumerate(lists):
            for pos, (b, e) in enumerate(zip(bits, E)):
                seen.setdefault(tuple(b), (e, r, pos))
        union = sorted(seen.items(), key=lambda kv: kv[1])[: K + 1]
        J, h = I.instance("gaussian", n, seed=70, inst=i)
        ref = O.qi_multi_search(J, h, K, iters, I.random_states(n, R, seed=71, inst=i))
        assert ref["count"] == len(union)
        for qpos, (tx, (e, r, pos)) in enumerate(union):
            assert tuple(ref["bits"][qpos].tolist()) == tx
            assert ref["E"][qpos] == e
            assert int(ref["src"][qpos]) == (r << 32) | pos
