"""The fused search kernel (one block per search through every iteration of a qis_iterate
call) against the per-kernel form of the same iteration (pair_scan 3: pick, fields, bound, scan
and merge as separate kernels every iteration) and against the oracle.

Both forms run the same arithmetic, so every kept list must be identical bit for bit (states,
energies, stamps, used flags), and so must the count of candidates decided. The cases cover the three flip sets, both exact modes, several instance sizes in
one context, iteration counts split over several calls, the full-fields fallback inside the
kernel (a ring of two parents, so most generators are gone), the survivor set held in global
memory (a smaller shared-memory allowance), and a +-J instance with massive ties."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2010_00180_gb300 import build, inputs as I, qis

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    qis.load()


def run(prec, ens, flips, ns, K, R, chunks, seed, pair_scan):
    ctx = qis.Context(K=K, R=R, precision=prec, max_n=max(ns), max_instances=len(ns), flips=flips)
    data = [I.instance(ens, n, seed=seed, inst=k) for k, n in enumerate(ns)]
    phis = [I.random_states(n, R, seed=seed + 1, inst=k) for k, n in enumerate(ns)]
    ctx.create_instances(data)
    for k in range(len(ns)):
        ctx.init_states(k, phis[k])
    ctx.set_tuning(pair_scan=pair_scan)
    for c in chunks:
        ctx.iterate(c)
    lists = [[ctx.search_list(k, r) for r in range(R)] for k in range(len(ns))]
    tops = [ctx.topk_states(k, K + 1) for k in range(len(ns))]
    counters = (ctx.candidate_count(), ctx.evaluated_pairs(), ctx.survivor_count())
    ctx.close()
    return data, phis, lists, tops, counters


def same(a, b):
    for la, lb in zip(a, b):
        for x, y in zip(la, lb):
            for key in ("count", "bits", "E", "stamp", "used"):
                assert np.array_equal(x[key], y[key]), key


CASES = [("split_bf16", "gaussian", "single_pair", [600, 130, 64], 120, 8),
         ("pm1_fp8", "pm1", "single_pair", [1024, 333], 120, 6),
         ("split_bf16", "uniform", "exchange", [300, 171], 40, 8),
         ("pm1_fp8", "pm1", "exchange", [200], 30, 8),
         ("split_bf16", "gaussian", "single", [1000, 77], 60, 8)]


@pytest.mark.parametrize("prec,ens,flips,ns,K,R", CASES)
def test_fused_equals_per_kernel_form(prec, ens, flips, ns, K, R):
    chunks = [1, 6, 1, 17]   # 25 iterations in calls of several lengths
    fused = run(prec, ens, flips, ns, K, R, chunks, 700, 1)
    single = run(prec, ens, flips, ns, K, R, [sum(chunks)], 700, 3)
    same(fused[2], single[2])
    for a, b in zip(fused[3], single[3]):
        assert np.array_equal(a["bits"], b["bits"]) and np.array_equal(a["E"], b["E"])
    # the candidates are fixed by the lists; the counts of pairs tested one by one and of
    # survivors are not: the order of the columns inside a bucket comes from shared-memory
    # atomics, a pair of two live rows of one bucket is tested in whichever row comes first, and
    # a pair at the filter band's edge can pass in one row's rounding and not the other's (the
    # merge decides every survivor exactly, so the lists never depend on it)
    assert fused[4][0] == single[4][0]
    data, phis = fused[0], fused[1]
    fl = {"single_pair": 0, "single": 1, "exchange": 2}[flips]
    J, h = data[0]
    for r in (0, R - 1):
        ref = O.qi_search(J, h, K, sum(chunks), phis[0][r], flips=fl)
        c = ref["count"]
        got = fused[2][0][r]
        assert np.array_equal(got["bits"], ref["bits"][:c]) and np.array_equal(got["stamp"], ref["stamp"][:c])


def test_fused_full_fields_fallback(monkeypatch):
    """A two-parent ring: a parent generated more than one iteration back finds no stored
    fields and the kernel sums its fields from scratch; the lists still equal the oracle's."""
    monkeypatch.setenv("QIS_FIELD_RING", "2")
    ns, K, R, iters = [257, 90], 30, 6, 20
    data, phis, lists, _, _ = run("split_bf16", "gaussian", "single_pair", ns, K, R, [iters], 710, 1)
    for k, (J, h) in enumerate(data):
        for r in range(R):
            ref = O.qi_search(J, h, K, iters, phis[k][r])
            c = ref["count"]
            got = lists[k][r]
            assert got["count"] == c
            for key in ("bits", "E", "used", "stamp"):
                assert np.array_equal(got[key], ref[key][:c]), (k, r, key)


def test_fused_survivors_in_global_memory_with_ties(monkeypatch):
    """+-J couplings (many equal energies at the threshold) with the shared-memory allowance of
    kept candidates lowered to 32: most iterations take the global-memory path of the merge."""
    monkeypatch.setenv("QIS_MERGE_SMEM_CAND", "32")
    ns, K, R, iters = [150], 60, 4, 25
    data, phis, lists, _, _ = run("pm1_fp8", "pm1", "single_pair", ns, K, R, [iters], 720, 1)
    J, h = data[0]
    for r in range(R):
        ref = O.qi_search(J, h, K, iters, phis[0][r])
        c = ref["count"]
        for key in ("bits", "E", "used", "stamp"):
            assert np.array_equal(lists[0][r][key], ref[key][:c]), (r, key)


def test_fused_runs_every_iteration_in_one_launch():
    """One qis_iterate call of the fused form is four launches (pick, field update, field GEMM,
    search kernel), whatever the number of iterations."""
    n, K, R = 200, 30, 4
    ctx = qis.Context(K=K, R=R, precision="split_bf16", max_n=n)
    J, h = I.instance("gaussian", n, seed=730)
    ctx.create_instance(J, h)
    ctx.init_states(0, I.random_states(n, R, seed=731))
    ctx.iterate(3)
    l0 = ctx.kernel_launches()
    ctx.iterate(40)
    assert ctx.kernel_launches() - l0 == 4
    ctx.close()


@pytest.mark.parametrize("prec,ens", [("split_bf16", "gaussian"), ("pm1_fp8", "pm1")])
def test_initial_energies_formed_by_the_first_iteration(prec, ens):
    """When qis_iterate starts the searches, E(psi0) is formed by the fused kernel from the exact
    fields of the first iteration ((sum_i s_i f_i + sum_i s_i h_i) / 2, Eq. 1); any other entry
    point, or a start whose energies are already known, takes them from the rescoring kernel.
    Every path must give E(psi0) of the oracle exactly (grid inputs: FP64 energies are exact),
    and the searches must equal the oracle's, across resets, new initial states and queries
    made before any iteration. (After one iteration psi0 has usually left the list: every
    kept energy is then E(psi0) + dE, so the list equality checks E(psi0).)"""
    n, K, R = 300, 30, 8
    J, h = I.instance(ens, n, seed=21)
    phi = I.random_states(n, R, seed=22)
    E0 = O.energies(J, h, phi)
    ctx = qis.Context(K=K, R=R, precision=prec, max_n=n, max_instances=1)
    ctx.create_instance(J, h)

    def psi0_energies():
        out = []
        for r in range(R):
            lst = ctx.search_list(0, r)
            k = np.flatnonzero(lst["stamp"] == 0)
            assert len(k) == 1
            assert np.array_equal(lst["bits"][k[0]], phi[r])
            out.append(lst["E"][k[0]])
        return np.array(out)

    def equals_oracle(iters):
        for r in range(R):
            got = ctx.search_list(0, r)
            ref = O.qi_search(J, h, K, iters, phi[r])
            c = ref["count"]
            assert got["count"] == c
            for key in ("bits", "E", "stamp", "used"):
                assert np.array_equal(got[key], ref[key][:c]), key

    ctx.init_states(0, phi)
    ctx.iterate(1)                      # started by qis_iterate: energies from the first iteration
    equals_oracle(1)                    # every new state's energy is E(psi0) + dE
    ctx.reset()
    assert np.array_equal(psi0_energies(), E0)   # started by a query: the rescoring kernel
    ctx.iterate(4)                      # the same searches continue (energies known)
    equals_oracle(4)
    ctx.reset()
    ctx.iterate(0)                      # no iteration: started without deferring
    assert np.array_equal(psi0_energies(), E0)
    ctx.init_states(0, phi)             # new initial states, then several calls
    ctx.iterate(2)
    ctx.iterate(3)
    equals_oracle(5)
    ctx.reset()
    ctx.iterate(5)
    equals_oracle(5)
    ctx.close()
