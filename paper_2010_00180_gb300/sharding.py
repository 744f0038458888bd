"""Several processes (one per GPU) running the QI search: which process runs which searches,
and the gather of kept lists to the owner of an instance for the Alg. 4 merge.

The R searches of an instance are independent until the Alg. 4 merge: each starts from its
own initial state and shares nothing with the others. So the work is split without any
communication during the iterations:

  * whole instances first: with at least as many instances as processes, process k runs
    all R searches of a contiguous block of instances and merges them itself;
  * with fewer instances than processes, every instance gets a group of processes and its
    R searches are split into contiguous ranges r0 <= r < r1 over the group.

The only exchange is at the end, for split instances: each process sends the kept lists of
its searches (R x (K+1) states, ~0.7 MB per n = 600 instance at K = 120, R = 64) to the
owner (the process that runs search 0), which imports them in search order and runs the
device merge (`qis_set_search_list` + `qis_merge`). Search r uses initial state r of the
instance wherever it runs, so the result is the single-process result exactly.
"""
from __future__ import annotations

from dataclasses import dataclass
from datetime import timedelta

import numpy as np


@dataclass(frozen=True)
class Shard:
    instance: int
    r0: int      # searches r0 <= r < r1 of the instance
    r1: int


def plan(n_instances: int, R: int, world: int) -> list[list[Shard]]:
    """Shards of every process (index = rank). Every (instance, r) appears exactly once."""
    if n_instances < 0 or R < 1 or world < 1:
        raise ValueError("need n_instances >= 0, R >= 1, world >= 1")
    out: list[list[Shard]] = [[] for _ in range(world)]
    if n_instances >= world:
        for k in range(world):
            lo, hi = k * n_instances // world, (k + 1) * n_instances // world
            out[k] = [Shard(i, 0, R) for i in range(lo, hi)]
        return out
    for i in range(n_instances):
        group = [k for k in range(world) if k % n_instances == i]
        g = len(group)
        for q, k in enumerate(group):
            r0, r1 = q * R // g, (q + 1) * R // g
            if r1 > r0:
                out[k].append(Shard(i, r0, r1))
    return out


def owner(shards: list[list[Shard]], instance: int) -> int:
    """Rank that runs search 0 of `instance` (it merges the instance's lists)."""
    for k, mine in enumerate(shards):
        for s in mine:
            if s.instance == instance and s.r0 == 0:
                return k
    raise KeyError(instance)


def split_instances(shards: list[list[Shard]]) -> set[int]:
    """Instances whose searches run on more than one process."""
    seen: dict[int, int] = {}
    for k, mine in enumerate(shards):
        for s in mine:
            seen[s.instance] = seen.get(s.instance, 0) + 1
    return {i for i, c in seen.items() if c > 1}


class PeerLost(RuntimeError):
    """A process of the run did not reach a step (it raised, exited or never joined)."""

    def __init__(self, step: int, missing: list[int]):
        super().__init__(f"step {step}: rank(s) {missing} did not arrive")
        self.step = step
        self.missing = missing


def check_peers(store, step: int, rank: int, world: int, timeout_s: float = 10.0) -> None:
    """Host-side liveness check between steps, before the next launch or collective: every
    process announces `step` in the key-value store (torch.distributed.TCPStore or any store
    with set/wait/check), then waits at most `timeout_s` for every other process's announcement.
    Raises PeerLost naming the processes that never announced (a process that left between
    steps), so the survivors stop instead of blocking in a collective that cannot complete."""
    keys = [f"qis/alive/{step}/{k}" for k in range(world)]
    store.set(keys[rank], "1")
    try:
        store.wait(keys, timedelta(seconds=timeout_s))
    except Exception:   # timeout, or the store's server process itself is gone
        missing = []
        for k, key in enumerate(keys):
            try:
                if not store.check([key]):
                    missing.append(k)
            except Exception:
                missing.append(k)
        raise PeerLost(step, missing or [k for k in range(world) if k != rank]) from None


def gather_lists(local: dict, shards: list[list[Shard]], rank: int, group=None) -> dict:
    """Collect the kept lists of split instances on their owners.

    local: {(instance, r): (bits (count, W) uint64, E (count,) float64)} of this process's
    searches of split instances (other entries are ignored). Returns, on each owner,
    {instance: [(bits, E) for r = 0..R-1]} for the split instances it owns (empty elsewhere).
    Uses one all_gather_object over the process group (gloo or NCCL)."""
    import torch.distributed as dist

    split = split_instances(shards)
    mine = {key: (np.asarray(b, np.uint64), np.asarray(e, np.float64))
            for key, (b, e) in local.items() if key[0] in split}
    world = dist.get_world_size(group)
    everyone = [None] * world
    dist.all_gather_object(everyone, mine, group=group)
    out: dict = {}
    for inst in sorted(split):
        if owner(shards, inst) != rank:
            continue
        R = max(s.r1 for mine_k in shards for s in mine_k if s.instance == inst)
        lists = []
        for r in range(R):
            src = next(k for k, mk in enumerate(shards) for s in mk if s.instance == inst and s.r0 <= r < s.r1)
            lists.append(everyone[src][(inst, r)])
        out[inst] = lists
    return out


def run_local(instances, states, shards_of_rank: list[Shard], K: int, iters: int, precision: str = "split_bf16",
              device: int = 0, **ctx_kw):
    """Run this process's searches on its GPU.

    instances: [(J, h)] of all instances; states: [R x W initial states] per instance.
    Returns (ctx, ids, lists): the context, {instance: local instance id}, and the kept lists
    {(instance, r): (bits, E)} of every search run here."""
    from . import qis as Q

    if not shards_of_rank:
        return None, {}, {}
    L = {s.r1 - s.r0 for s in shards_of_rank}
    if len(L) != 1:
        raise ValueError("every shard of one process must cover the same number of searches")
    Rl = L.pop()
    max_n = max(np.asarray(instances[s.instance][1]).shape[0] for s in shards_of_rank)
    ctx = Q.Context(K=K, R=Rl, precision=precision, max_n=max_n, max_instances=len(shards_of_rank),
                    device=device, **ctx_kw)
    ids = {}
    for s in shards_of_rank:
        J, h = instances[s.instance]
        iid = ctx.create_instance(J, h)
        ctx.init_states(iid, np.asarray(states[s.instance])[s.r0:s.r1])
        ids[s.instance] = iid
    ctx.iterate(iters)
    lists = {}
    for s in shards_of_rank:
        for r in range(s.r0, s.r1):
            lst = ctx.search_list(ids[s.instance], r - s.r0)
            lists[(s.instance, r)] = (lst["bits"], lst["E"])
    return ctx, ids, lists


def merge_gathered(instances, states, gathered: dict, K: int, precision: str = "split_bf16", device: int = 0,
                   k: int | None = None) -> dict:
    """Alg. 4 merge on this GPU of the gathered lists of each owned split instance.
    Returns {instance: topk dict (bits, E, src, count)}."""
    from . import qis as Q

    out = {}
    for inst, lists in sorted(gathered.items()):
        J, h = instances[inst]
        n = np.asarray(h).shape[0]
        ctx = Q.Context(K=K, R=len(lists), precision=precision, max_n=n, max_instances=1, device=device)
        try:
            ctx.create_instance(J, h)
            ctx.init_states(0, np.asarray(states[inst])[: len(lists)])
            for r, (bits, E) in enumerate(lists):
                ctx.set_search_list(0, r, bits, E)
            out[inst] = ctx.topk_states(0, K + 1 if k is None else k)
        finally:
            ctx.close()
    return out
