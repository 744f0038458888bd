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


def _leaver(rank, world, port, steps_of_rank, q):
    """A gloo process group over a host TCPStore; each step is the liveness check and then a
    collective. Rank `rank` runs steps 0 .. steps_of_rank[rank] - 1 and then leaves (a process
    that exits between steps, with nothing in flight); a rank that does not leave reports the
    PeerLost it gets at the liveness check, before it would enter a collective that cannot
    complete."""
    done = 0
    try:
        sys.path.insert(0, ROOT)
        import datetime
        import torch
        import torch.distributed as dist
        from paper_2010_00180_gb300 import sharding as S
        store = dist.TCPStore("127.0.0.1", port, world, rank == 0, timeout=datetime.timedelta(seconds=30),
                              wait_for_workers=False)
        dist.init_process_group("gloo", store=store, rank=rank, world_size=world,
                                timeout=datetime.timedelta(seconds=30))
        for step in range(steps_of_rank[rank]):
            S.check_peers(store, step, rank, world, timeout_s=3.0)
            x = torch.ones(1)
            dist.all_reduce(x)                  # the step's exchange
            assert x.item() == world
            done += 1
        q.put((rank, done, None))
        if rank == 0:                           # the store's server stays up until the others are done
            import time
            time.sleep(5.0)
    except Exception as e:
        q.put((rank, done, e.missing if hasattr(e, "missing") else repr(e)))


def test_a_rank_that_leaves_between_steps_is_reported_not_waited_for():
    """World size 2 on CPU with gloo: rank 1 takes part in steps 0 and 1 (check and all_reduce)
    and exits; rank 0 reaches step 2, where the host liveness check raises PeerLost naming rank 1
    within its 3 s timeout instead of blocking in the all_reduce."""
    import multiprocessing as mp
    import time
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    steps = {0: 5, 1: 2}
    t0 = time.time()
    ps = [ctx.Process(target=_leaver, args=(k, world, port, steps, q)) for k in range(world)]
    for p in ps:
        p.start()
    out = {}
    for _ in range(world):
        rank, done, err = q.get(timeout=120)
        out[rank] = (done, err)
    for p in ps:
        p.join(timeout=60)
    assert out[1] == (2, None)                 # left after its two steps, no error of its own
    assert out[0] == (2, [1])                  # rank 0 stopped at step 2, naming rank 1
    assert time.time() - t0 < 60
