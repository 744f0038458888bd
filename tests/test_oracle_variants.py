"""Pins of the oracle's flip-set variants (Sec. V outlook): single flips only (J = 1) and
spin exchanges only (the XX + YY interaction, magnetisation conserving).

Checked against facts independent of the oracle: numpy energies of Eq. (1), an order-
statistics restatement of Alg. 2-3 whose candidate set is built here from the definition,
magnetisation conservation, and the special case where the list holds every reachable
state (the whole spectrum for J = 1, the whole magnetisation sector for exchanges).
"""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2010_00180_gb300 import inputs as I

SINGLES, EXCHANGE = 1, 2
ENSEMBLES = ["gaussian", "uniform", "pm1"]


def spins_of(bits, n):
    return 1.0 - 2.0 * I.unpack_bits(bits, n).astype(np.float64)


def energy_np(J, h, S):
    U = np.triu(J, 1)
    return np.einsum("mi,ij,mj->m", S, U, S) + S @ h


def variant_candidates(bits, n, flips):
    """(c, flipped sites) of one state for a flip set, in candidate order, from the
    definition: singles c = i; pairs c = n + rank(i, j); an exchange needs s_i != s_j."""
    s = spins_of(bits, n)[0]
    out = []
    if flips != EXCHANGE:
        out += [(i, (i,)) for i in range(n)]
    if flips != SINGLES:
        for c, (i, j) in enumerate(itertools.combinations(range(n), 2)):
            if flips == EXCHANGE and s[i] == s[j]:
                continue
            out.append((n + c, (i, j)))
    return out


def apply(bits, sites):
    x = np.asarray(bits, np.uint64).reshape(-1).copy()
    for i in sites:
        x[i // 64] ^= np.uint64(1) << np.uint64(i % 64)
    return x


def batch_model(J, h, K, I_, psi0, flips):
    """Alg. 2-3 as order statistics over the variant's candidate set (numpy energies)."""
    n = h.shape[0]
    psi0 = np.asarray(psi0, np.uint64).reshape(-1)
    lst = [[energy_np(J, h, spins_of(psi0, n))[0], 0, tuple(int(w) for w in psi0), False]]
    for t in range(1, I_ + 1):
        k = next((q for q, e in enumerate(lst) if not e[3]), None)
        if k is None:
            continue
        lst[k][3] = True
        members = {e[2] for e in lst}
        parent = np.array(lst[k][2], np.uint64)
        new = []
        for c, sites in variant_candidates(parent, n, flips):
            x = apply(parent, sites)
            tx = tuple(int(w) for w in x)
            if tx not in members:
                new.append([energy_np(J, h, spins_of(x, n))[0], (t << 32) | c, tx, False])
        lst = sorted(lst + new, key=lambda e: (e[0], e[1]))[: K + 1]
    return lst


def assert_same_list(res, model):
    assert res["count"] == len(model)
    for q, (E, st, tx, used) in enumerate(model):
        assert res["E"][q] == E
        assert int(res["stamp"][q]) == st
        assert tuple(int(w) for w in res["bits"][q]) == tx
        assert bool(res["used"][q]) == used


@pytest.mark.parametrize("flips", [SINGLES, EXCHANGE])
@pytest.mark.parametrize("ens", ENSEMBLES)
@pytest.mark.parametrize("n,K,I_", [(5, 3, 9), (8, 10, 12), (11, 30, 25)])
def test_variants_equal_batch_model(flips, ens, n, K, I_):
    J, h = I.instance(ens, n, seed=121, inst=n * 10 + flips)
    for psi0 in I.random_states(n, 3, seed=122, inst=n):
        res = O.qi_search(J, h, K, I_, psi0, flips=flips)
        assert_same_list(res, batch_model(J, h, K, I_, psi0, flips))


@pytest.mark.parametrize("flips", [SINGLES, EXCHANGE])
@pytest.mark.parametrize("n", [7, 40])
def test_candidate_sets(flips, n):
    """Candidates outside the flip set are excluded (+inf); the rest equal the full set's."""
    J, h = I.instance("gaussian", n, seed=130, inst=n)
    b = I.random_states(n, 1, seed=131, inst=n)[0]
    full = O.candidates(J, h, b)
    var = O.candidates(J, h, b, flips=flips)
    keep = np.zeros(full.size, bool)
    keep[[c for c, _ in variant_candidates(b, n, flips)]] = True
    assert np.array_equal(var[keep], full[keep])
    assert np.all(np.isinf(var[~keep]))


@pytest.mark.parametrize("ens", ENSEMBLES)
def test_exchange_conserves_magnetisation(ens):
    n, K = 30, 40
    J, h = I.instance(ens, n, seed=140)
    for psi0 in I.random_states(n, 3, seed=141):
        res = O.qi_search(J, h, K, 40, psi0, flips=EXCHANGE)
        m0 = int(I.unpack_bits(psi0, n).sum())
        c = res["count"]
        assert np.all(I.unpack_bits(res["bits"][:c], n).sum(1) == m0)
        assert np.array_equal(res["E"][:c], energy_np(J, h, spins_of(res["bits"][:c], n)))


@pytest.mark.parametrize("ens", ["gaussian", "pm1"])
def test_exchange_full_sector_spectrum(ens):
    """K + 1 = C(n, m) and I >= C(n, m): the list is the whole magnetisation sector of the
    initial state in key order (exchanges connect every state of a sector)."""
    n, m = 8, 3
    J, h = I.instance(ens, n, seed=150)
    sector = [sum(1 << i for i in c) for c in itertools.combinations(range(n), m)]
    size = len(sector)
    assert size == math.comb(n, m)
    psi0 = np.array([sector[5]], np.uint64)
    res = O.qi_search(J, h, size - 1, size, psi0, flips=EXCHANGE)
    S = 1.0 - 2.0 * ((np.array(sector, np.uint64)[:, None] >> np.arange(n, dtype=np.uint64)) & np.uint64(1))
    E = energy_np(J, h, S.astype(np.float64))
    assert res["count"] == size and res["used"].all()
    assert np.array_equal(res["E"], np.sort(E))
    assert sorted(int(b) for b in res["bits"][:, 0]) == sorted(sector)
    assert_same_list(res, batch_model(J, h, size - 1, size, psi0, EXCHANGE))


def test_exchange_sector_smaller_than_list_ends_the_search():
    """With one up spin the sector has n states; a longer list just stops filling."""
    n, K = 6, 10
    J, h = I.instance("gaussian", n, seed=151)
    psi0 = np.array([1 << 2], np.uint64)
    res = O.qi_search(J, h, K, 30, psi0, flips=EXCHANGE)
    assert res["count"] == n and res["used"][:n].all() and res["productive"] == n
    assert sorted(int(b) for b in res["bits"][:n, 0]) == [1 << i for i in range(n)]


@pytest.mark.parametrize("ens", ["gaussian", "pm1"])
@pytest.mark.parametrize("n", [4, 6])
def test_singles_full_spectrum(ens, n):
    """J = 1 with K + 1 = 2^N and I >= 2^N: the whole spectrum (single flips connect all)."""
    J, h = I.instance(ens, n, seed=160, inst=n)
    K = 2 ** n - 1
    psi0 = I.random_states(n, 1, seed=161, inst=n)[0]
    res = O.qi_search(J, h, K, 2 ** n, psi0, flips=SINGLES)
    S = 1.0 - 2.0 * ((np.arange(2 ** n, dtype=np.uint64)[:, None] >> np.arange(n, dtype=np.uint64)) & np.uint64(1))
    assert res["count"] == 2 ** n and res["used"].all()
    assert np.array_equal(res["E"], np.sort(energy_np(J, h, S.astype(np.float64))))


@pytest.mark.parametrize("flips", [SINGLES, EXCHANGE])
@pytest.mark.parametrize("ens", ENSEMBLES)
def test_one_iteration_closed_form(flips, ens):
    n, K = 20, 60
    J, h = I.instance(ens, n, seed=170)
    psi0 = I.random_states(n, 1, seed=171)[0]
    res = O.qi_search(J, h, K, 1, psi0, flips=flips)
    E0 = energy_np(J, h, spins_of(psi0, n))[0]
    keys = [(E0, -1, psi0)]
    for c, sites in variant_candidates(psi0, n, flips):
        x = apply(psi0, sites)
        keys.append((energy_np(J, h, spins_of(x, n))[0], c, x))
    keys.sort(key=lambda k: (k[0], k[1]))
    keys = keys[: K + 1]
    assert res["count"] == len(keys)
    for q, (E, c, x) in enumerate(keys):
        assert res["E"][q] == E and np.array_equal(res["bits"][q], x)
        assert int(res["stamp"][q]) == (0 if c < 0 else (1 << 32) | c)


@pytest.mark.parametrize("flips", [SINGLES, EXCHANGE])
def test_multi_search_variant_is_topk_of_union(flips):
    n, K, L = 12, 20, 5
    J, h = I.instance("gaussian", n, seed=180)
    phi = I.random_states(n, L, seed=181)
    res = O.qi_multi_search(J, h, K, K, phi, per_search=True, flips=flips)
    seen = {}
    for r, s in enumerate(res["searches"]):
        ref = O.qi_search(J, h, K, K, phi[r], flips=flips)
        assert np.array_equal(ref["E"], s["E"]) and np.array_equal(ref["bits"], s["bits"])
        for pos in range(s["count"]):
            seen.setdefault(tuple(s["bits"][pos].tolist()), (s["E"][pos], r, pos))
    union = sorted(seen.items(), key=lambda kv: kv[1])[: K + 1]
    assert res["count"] == len(union)
    for q, (tx, (E, r, pos)) in enumerate(union):
        assert tuple(res["bits"][q].tolist()) == tx and res["E"][q] == E
