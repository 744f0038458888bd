"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test checks the oracle (oracle/qis_oracle.c) against mathematics the paper fixes:
  * Eq. (1) evaluated independently with numpy (exact on the grid inputs, whose every
    partial sum is an exact FP64 number),
  * 2^N brute-force enumeration done with numpy,
  * the special case K + 1 = 2^N, where the method must return the full sorted spectrum,
  * a one-iteration closed form, list invariants and a neighbour-closure property,
  * an independent batch formulation of Alg. 2-3 (the order-statistics reading used by
    the GPU: top-(K+1) by (E, stamp) of the old list and the new non-duplicate
    candidates), and the top-(K+1) reading of the Alg. 4 merge.
"""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_2010_00180_gb300 import inputs as I


def spins_of(bits, n):
    return 1.0 - 2.0 * I.unpack_bits(bits, n).astype(np.float64)


def energy_np(J, h, S):
    """Eq. (1) for each row of S (m, n) of +-1 spins, written with numpy."""
    U = np.triu(J, 1)
    return np.einsum("mi,ij,mj->m", S, U, S) + S @ h


def flips(n):
    """The flip sets of Sec. III in candidate order: singles (i,), then pairs (i, j), i < j."""
    return [(i,) for i in range(n)] + list(itertools.combinations(range(n), 2))


def flipped_states(bits, n):
    bits = np.asarray(bits, np.uint64).reshape(-1)
    out = []
    for f in flips(n):
        x = bits.copy()
        for i in f:
            x[i // 64] ^= np.uint64(1) << np.uint64(i % 64)
        out.append(x)
    return np.array(out)


def all_states(n):
    psi = np.arange(2 ** n, dtype=np.uint64)
    return psi, 1.0 - 2.0 * ((psi[:, None] >> np.arange(n, dtype=np.uint64)) & np.uint64(1)).astype(np.float64)


ENSEMBLES = ["gaussian", "uniform", "pm1"]


@pytest.mark.parametrize("ens", ENSEMBLES)
@pytest.mark.parametrize("n", [2, 5, 16, 70, 130])
def test_energy_is_eq1(ens, n):
    J, h = I.instance(ens, n, seed=11, inst=n)
    st = I.random_states(n, 6, seed=5, inst=n)
    got = O.energies(J, h, st)
    want = energy_np(J, h, spins_of(st, n))
    assert np.array_equal(got, want)   # exact: grid inputs make every partial sum exact


@pytest.mark.parametrize("ens", ENSEMBLES)
@pytest.mark.parametrize("n", [2, 7, 16, 67])
def test_candidate_energies_equal_flipped_state_energies(ens, n):
    J, h = I.instance(ens, n, seed=3, inst=n)
    for st in I.random_states(n, 3, seed=9, inst=n):
        got = O.candidates(J, h, st)
        want = energy_np(J, h, spins_of(flipped_states(st, n), n))
        assert got.shape == (n * (n + 1) // 2,)
        assert np.array_equal(got, want)


def test_candidate_energies_non_grid_inputs():
    """Off the grid the incremental update still matches Eq. (1) to rounding."""
    n = 40
    rng = np.random.default_rng(0)
    A = rng.standard_normal((n, n))
    J = np.triu(A, 1) + np.triu(A, 1).T
    h = rng.standard_normal(n)
    st = I.random_states(n, 1, seed=1)[0]
    got = O.candidates(J, h, st)
    want = energy_np(J, h, spins_of(flipped_states(st, n), n))
    assert np.allclose(got, want, rtol=1e-12, atol=1e-11)


def test_fields_and_pair_rank():
    n = 33
    J, h = I.instance("gaussian", n, seed=1)
    st = I.random_states(n, 1, seed=2)[0]
    s = spins_of(st, n)[0]
    assert np.array_equal(O.fields(J, h, st), J @ s + h)
    c = n
    for i in range(n):
        for j in range(i + 1, n):
            assert O.pair_rank(n, i, j) == c - n
            c += 1


@pytest.mark.parametrize("ens", ["gaussian", "pm1"])
@pytest.mark.parametrize("n", [6, 12])
def test_brute_force_matches_enumeration(ens, n):
    J, h = I.instance(ens, n, seed=4)
    psi, S = all_states(n)
    E = energy_np(J, h, S)
    order = np.lexsort((psi, E))
    k = 20
    bpsi, bE = O.brute_force(J, h, k)
    assert np.array_equal(bE, E[order[:k]])
    assert np.array_equal(bpsi, psi[order[:k]])


def test_n16_ground_state_by_brute_force():
    """N=16 Gaussian instance, seed 0, K=8 kept (+1 slot), R=4 random initial states, I=K."""
    n, K, R = 16, 8, 4
    J, h = I.instance("gaussian", n, seed=0)
    phi = I.random_states(n, R, seed=0)
    res = O.qi_multi_search(J, h, K, K, phi, per_search=True)
    psi, S = all_states(n)
    E = energy_np(J, h, S)
    gs = int(np.argmin(E))
    # every kept energy equals Eq. (1) of its state
    assert res["count"] == K + 1
    assert np.array_equal(res["E"], energy_np(J, h, spins_of(res["bits"], n)))
    for s in res["searches"]:
        assert np.array_equal(s["E"][: s["count"]], energy_np(J, h, spins_of(s["bits"][: s["count"]], n)))
    # this seeded instance: the merged list holds the exact K+1 lowest states
    assert int(res["bits"][0, 0]) == gs
    assert np.array_equal(res["E"], np.sort(E)[: K + 1])


# ---------------------------------------------------------------- batch model
def batch_model(J, h, K, I_, psi0):
    """Alg. 2-3 restated as order statistics: each iteration keeps the K+1 smallest keys
    (E, stamp) of (old list) + (candidates not in the old list); stamp = (t << 32) | c.
    Energies come from numpy's Eq. (1), not from the oracle."""
    n = h.shape[0]
    psi0 = np.asarray(psi0, np.uint64).reshape(-1)
    E0 = energy_np(J, h, spins_of(psi0, n))[0]
    lst = [[E0, 0, tuple(int(w) for w in psi0), False]]
    for t in range(1, I_ + 1):
        k = next((q for q, e in enumerate(lst) if not e[3]), None)
        if k is None:
            continue
        lst[k][3] = True
        members = {e[2] for e in lst}
        fs = flipped_states(np.array(lst[k][2], np.uint64), n)
        Ec = energy_np(J, h, spins_of(fs, n))
        new = []
        for c, x in enumerate(fs):
            tx = tuple(int(w) for w in x)
            if tx not in members:
                new.append([Ec[c], (t << 32) | c, tx, False])
        lst = sorted(lst + new, key=lambda e: (e[0], e[1]))[: K + 1]
    return lst


def assert_same_list(res, model, n):
    assert res["count"] == len(model)
    for q, (E, st, tx, used) in enumerate(model):
        assert res["E"][q] == E
        assert int(res["stamp"][q]) == st
        assert tuple(int(w) for w in res["bits"][q]) == tx
        assert bool(res["used"][q]) == used


@pytest.mark.parametrize("ens", ENSEMBLES)
@pytest.mark.parametrize("n,K,I_", [(3, 2, 5), (5, 1, 4), (5, 3, 9), (8, 10, 12), (11, 40, 30), (12, 7, 25)])
def test_sequential_equals_batch_model(ens, n, K, I_):
    J, h = I.instance(ens, n, seed=21, inst=n * 100 + K)
    for psi0 in I.random_states(n, 3, seed=22, inst=n):
        res = O.qi_search(J, h, K, I_, psi0)
        assert_same_list(res, batch_model(J, h, K, I_, psi0), n)


@pytest.mark.parametrize("ens", ["gaussian", "pm1"])
@pytest.mark.parametrize("n", [3, 5, 8])
def test_full_spectrum_when_list_holds_every_state(ens, n):
    """K + 1 = 2^N and I >= 2^N: the list ends as the whole spectrum in key order."""
    J, h = I.instance(ens, n, seed=8, inst=n)
    K = 2 ** n - 1
    psi0 = I.random_states(n, 1, seed=7, inst=n)[0]
    res = O.qi_search(J, h, K, 2 ** n, psi0)
    psi, S = all_states(n)
    E = energy_np(J, h, S)
    assert res["count"] == 2 ** n
    assert np.array_equal(res["E"], np.sort(E))
    assert sorted(int(b) for b in res["bits"][:, 0]) == list(range(2 ** n))
    assert res["used"].all() and res["productive"] == 2 ** n
    # ties (pm1 has many) are ordered by arrival
    for q in range(1, 2 ** n):
        if res["E"][q] == res["E"][q - 1]:
            assert res["stamp"][q] > res["stamp"][q - 1]
    assert_same_list(res, batch_model(J, h, K, 2 ** n, psi0), n)


@pytest.mark.parametrize("ens", ENSEMBLES)
@pytest.mark.parametrize("n,K", [(6, 4), (10, 30), (20, 120), (70, 25)])
def test_one_iteration_closed_form(ens, n, K):
    """After one iteration: the first K+1 of {phi} + all its flips by (E, c)."""
    J, h = I.instance(ens, n, seed=30, inst=n)
    psi0 = I.random_states(n, 1, seed=31, inst=n)[0]
    res = O.qi_search(J, h, K, 1, psi0)
    fs = flipped_states(psi0, n)
    E0 = energy_np(J, h, spins_of(psi0, n))[0]
    Ec = energy_np(J, h, spins_of(fs, n))
    keys = [(E0, -1)] + [(Ec[c], c) for c in range(len(fs))]
    keys.sort()
    keys = keys[: K + 1]
    assert res["count"] == len(keys)
    for q, (E, c) in enumerate(keys):
        assert res["E"][q] == E
        want = psi0 if c < 0 else fs[c]
        assert np.array_equal(res["bits"][q], want)
        assert int(res["stamp"][q]) == (0 if c < 0 else (1 << 32) | c)


@pytest.mark.parametrize("ens", ENSEMBLES)
def test_invariants_over_iterations(ens):
    n, K = 24, 30
    J, h = I.instance(ens, n, seed=40)
    psi0 = I.random_states(n, 1, seed=41)[0]
    last_T = np.inf
    for t in range(1, 40):
        res = O.qi_search(J, h, K, t, psi0)
        c = res["count"]
        E = res["E"][:c]
        assert np.all(np.diff(E) >= 0)                                  # sorted
        assert len({tuple(b) for b in res["bits"][:c].tolist()}) == c   # distinct
        # one parent per iteration until every kept state has been used (then nothing changes)
        assert res["productive"] == t or (res["productive"] < t and res["used"][:c].all())
        assert int(res["used"].sum()) <= res["productive"]   # a used parent may be evicted later
        assert np.array_equal(E, energy_np(J, h, spins_of(res["bits"][:c], n)))
        T = res["E"][K] if c == K + 1 else np.inf
        assert T <= last_T                                              # threshold never rises
        last_T = T


@pytest.mark.parametrize("ens", ENSEMBLES)
def test_neighbour_closure_of_used_states(ens):
    """Every flip of a used state is in the list or not below the last slot's energy."""
    n, K, I_ = 18, 20, 15
    J, h = I.instance(ens, n, seed=50)
    psi0 = I.random_states(n, 1, seed=51)[0]
    res = O.qi_search(J, h, K, I_, psi0)
    members = {tuple(b) for b in res["bits"].tolist()}
    T = res["E"][K]
    for q in range(K + 1):
        if not res["used"][q]:
            continue
        fs = flipped_states(res["bits"][q], n)
        Ec = energy_np(J, h, spins_of(fs, n))
        for x, e in zip(fs.tolist(), Ec):
            assert tuple(x) in members or e >= T


@pytest.mark.parametrize("ens", ENSEMBLES)
@pytest.mark.parametrize("n,K,L", [(8, 5, 4), (12, 20, 6), (20, 15, 5)])
def test_multi_search_merge_is_topk_of_union(ens, n, K, L):
    """Alg. 4 merge = first K+1 of the union of the L lists, each state at its first
    occurrence, ordered by (E, search index, position)."""
    J, h = I.instance(ens, n, seed=60, inst=n)
    phi = I.random_states(n, L, seed=61, inst=n)
    res = O.qi_multi_search(J, h, K, K, phi, per_search=True)
    seen = {}
    for r, s in enumerate(res["searches"]):
        ref = O.qi_search(J, h, K, K, phi[r])
        assert np.array_equal(ref["E"], s["E"]) and np.array_equal(ref["bits"], s["bits"])
        for pos in range(s["count"]):
            tx = tuple(s["bits"][pos].tolist())
            if tx not in seen:
                seen[tx] = (s["E"][pos], r, pos)
    union = sorted(seen.items(), key=lambda kv: kv[1])[: K + 1]
    assert res["count"] == len(union)
    for q, (tx, (E, r, pos)) in enumerate(union):
        assert tuple(res["bits"][q].tolist()) == tx
        assert res["E"][q] == E
        assert int(res["src"][q]) == (r << 32) | pos


def test_invalid_arguments():
    J, h = I.instance("gaussian", 3, seed=0)
    psi0 = I.random_states(3, 1, seed=0)[0]
    with pytest.raises(O.OracleError):
        O.qi_search(J, h, 8, 1, psi0)        # K < 2^N violated
    with pytest.raises(O.OracleError):
        O.qi_search(J, h, 0, 1, psi0)
    O.qi_search(J, h, 7, 20, psi0)           # K = 2^N - 1 is allowed


def test_uniform_ensemble_sanity_bands():
    """Sanity bands from Sec. IV on the paper's U[-1/2, 1/2] ensemble (not exact parity):
    <E_1> ~ -0.218 N^1.5 + 0.79, and the multi search with (I, K, L) = (N/2, K0, N)
    finds the ground state of (nearly) every instance."""
    n, n_inst = 14, 24
    K0 = n * (n + 1) // 2 + 1
    psi, S = all_states(n)
    gs_E, hits = [], 0
    for k in range(n_inst):
        J, h = I.instance("uniform", n, seed=70, inst=k)
        E = energy_np(J, h, S)
        gs_E.append(E.min())
        phi = I.random_states(n, n, seed=71, inst=k)
        res = O.qi_multi_search(J, h, K0, n // 2, phi)
        hits += res["E"][0] == E.min()
    fit = -0.218 * n ** 1.5 + 0.79
    assert abs(np.mean(gs_E) - fit) < 0.15 * abs(fit)
    assert hits >= n_inst - 1
