"""Energies from scratch (Eq. 1) when the rows of a group of states are split over several
blocks (few groups, large n): the exact integer form and the FP64 form equal numpy's energies,
the initial energies of the searches too, and the merged lists' energies are the same whether
one instance or every instance is asked for."""
import numpy as np
import pytest

from paper_2010_00180_gb300 import build, inputs as I, qis

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    qis.load()


def energy_np(J, h, S):
    return np.einsum("mi,ij,mj->m", S, np.triu(J, 1), S) + S @ h


def off_grid(n, seed):
    rng = np.random.default_rng(seed)
    J = np.triu(rng.standard_normal((n, n)), 1)
    return J + J.T, rng.standard_normal(n)


@pytest.mark.parametrize("count", [5, 40])
def test_split_rows_exact_form(count):
    """On-grid couplings (exact int64 sums), n = 1100: a few groups of 16 states, rows split."""
    n = 1100
    J, h = I.instance("gaussian", n, seed=450)
    ctx = qis.Context(K=8, R=2, precision="split_bf16", max_n=n, max_instances=1)
    ctx.create_instance(J, h)
    assert ctx.instance_info(0)[2] == 0
    bits = I.random_states(n, count, seed=451)
    S = 1.0 - 2.0 * I.unpack_bits(bits, n).astype(np.float64)
    assert np.array_equal(ctx.energies(0, bits), energy_np(J, h, S))
    ctx.close()


def test_split_rows_fp64_form():
    """Off-grid couplings (rounded for the search, rescored in FP64 over row parts)."""
    n = 1100
    J, h = off_grid(n, 452)
    ctx = qis.Context(K=8, R=2, precision="split_bf16", max_n=n, max_instances=1)
    ctx.create_instance(J, h)
    assert ctx.instance_info(0)[2] == 1
    bits = I.random_states(n, 20, seed=453)
    S = 1.0 - 2.0 * I.unpack_bits(bits, n).astype(np.float64)
    np.testing.assert_allclose(ctx.energies(0, bits), energy_np(J, h, S), rtol=1e-12, atol=1e-9)
    ctx.close()


def test_split_rows_initial_energies():
    """The searches' initial energies (16 states per block, rows split) equal numpy's."""
    n, R = 1100, 4
    J, h = I.instance("gaussian", n, seed=454)
    phi = I.random_states(n, R, seed=455)
    ctx = qis.Context(K=8, R=R, precision="split_bf16", max_n=n, max_instances=1, flips="single")
    ctx.create_instance(J, h)
    ctx.init_states(0, phi)
    S = 1.0 - 2.0 * I.unpack_bits(phi, n).astype(np.float64)
    ref = energy_np(J, h, S)
    for r in range(R):
        lst = ctx.search_list(0, r)
        assert lst["count"] == 1 and lst["E"][0] == ref[r]
    ctx.close()


def test_split_rows_merged_lists_agree():
    """An on-grid and an off-grid instance in one context: every merged energy is the same
    from qis_topk_states_all and from qis_topk_states, and near numpy's."""
    n, K, R, iters = 1100, 12, 3, 6
    data = [I.instance("gaussian", n, seed=456), off_grid(n, 457)]
    ctx = qis.Context(K=K, R=R, precision="split_bf16", max_n=n, max_instances=2, flips="single")
    ctx.create_instances(data)
    for k in range(2):
        ctx.init_states(k, I.random_states(n, R, seed=458, inst=k))
    ctx.iterate(iters)
    every = ctx.topk_states_all(K + 1)
    for k, (J, h) in enumerate(data):
        one = ctx.topk_states(k, K + 1)
        for key in ("count", "bits", "E", "src"):
            assert np.array_equal(every[k][key], one[key]), (k, key)
        S = 1.0 - 2.0 * I.unpack_bits(one["bits"][: one["count"]], n).astype(np.float64)
        np.testing.assert_allclose(one["E"][: one["count"]], energy_np(J, h, S), rtol=1e-12, atol=1e-9)
    ctx.close()
