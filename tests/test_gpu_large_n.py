"""Instances above 4096 spins (up to 16384): survivor entries with 14-bit sites, and above
n_pad = 8192 coupling digits of 11 bits (the FP32 partial sums of the digit GEMM stay exact).
The J = 1 variant (single flips only) is the one meant for such sizes (Sec. V outlook)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2010_00180_gb300 import build, inputs as I, qis

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    qis.load()


def grid_instance(n, seed, bits):
    """Uniform couplings (the paper's U[-1/2, 1/2]) rounded to the grid 2^-bits, so that the
    fixed-point grid holds them exactly at this size."""
    J, h = I.instance("uniform", n, seed=seed)
    s = float(2 ** bits)
    return np.round(J * s) / s, np.round(h * s) / s


def same(g, o, what=""):
    c = o["count"]
    assert g["count"] == c, what
    for key in ("bits", "E", "used", "stamp"):
        assert np.array_equal(g[key], o[key][:c]), (what, key)


def test_single_flips_n9000_eleven_bit_digits():
    n, K, R, iters = 9000, 12, 2, 6
    J, h = grid_instance(n, 500, 20)
    phi = I.random_states(n, R, seed=501)
    ctx = qis.Context(K=K, R=R, precision="split_bf16", max_n=n, max_instances=1, flips="single")
    ctx.create_instance(J, h)
    q, digits, rounded = ctx.instance_info(0)
    assert q == 20 and digits == 2 and not rounded   # two 11-bit digits hold 2^19 (|J| <= 1/2)
    ctx.init_states(0, phi)
    for t in range(1, iters + 1):
        ctx.iterate(1)
        if t in (2, iters):
            for r in range(R):
                same(ctx.search_list(0, r), O.qi_search(J, h, K, t, phi[r], flips=1), f"t={t} r={r}")
    ctx.close()


def test_pairs_n5000_wide_sites():
    n, K, R, iters = 5000, 8, 2, 3
    J, h = grid_instance(n, 510, 20)
    phi = I.random_states(n, R, seed=511)
    ctx = qis.Context(K=K, R=R, precision="split_bf16", max_n=n, max_instances=1)
    ctx.create_instance(J, h)
    ctx.init_states(0, phi)
    ctx.iterate(iters)
    for r in range(R):
        same(ctx.search_list(0, r), O.qi_search(J, h, K, iters, phi[r]), f"r={r}")
    top = ctx.topk_states(0, K + 1)
    ref = O.qi_multi_search(J, h, K, iters, phi)
    assert top["count"] == ref["count"]
    assert np.array_equal(top["bits"], ref["bits"][: ref["count"]])
    ctx.close()


def test_single_flips_maximum_size():
    """n = 16384, the largest instance a context takes (max_n): a few iterations equal the
    oracle."""
    n, K, R, iters = 16384, 8, 1, 3
    J, h = grid_instance(n, 520, 18)
    phi = I.random_states(n, R, seed=521)
    ctx = qis.Context(K=K, R=R, precision="split_bf16", max_n=n, max_instances=1, flips="single")
    ctx.create_instance(J, h)
    assert not ctx.instance_info(0)[2]
    ctx.init_states(0, phi)
    ctx.iterate(iters)
    same(ctx.search_list(0, 0), O.qi_search(J, h, K, iters, phi[0], flips=1))
    ctx.close()
    with pytest.raises(qis.QISError):
        qis.Context(K=K, R=R, precision="split_bf16", max_n=n + 1, max_instances=1)
