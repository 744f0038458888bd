"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Inputs are the seeded grid-valued ensembles, on which every energy is an exact FP64
number; the kept lists must then agree exactly: same states in the same order, same
energies (bitwise), same used flags, same stamps. Merged lists (Alg. 4) must agree in
states, source positions and FP64-rescored energies (1e-9 relative, the rescoring sums in
another order than the oracle).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2010_00180_gb300 import build, inputs as I, qis

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    qis.load()


def assert_list_equal(g, o, what=""):
    c = o["count"]
    assert g["count"] == c, what
    assert np.array_equal(g["bits"], o["bits"][:c]), what
    assert np.array_equal(g["E"], o["E"][:c]), what
    assert np.array_equal(g["used"], o["used"][:c]), what
    assert np.array_equal(g["stamp"], o["stamp"][:c]), what


def run_pair(ens, n, K, R, I_, precision, seed=0, n_inst=1, per_iter=False, sample=None):
    """Run the GPU on n_inst instances, compare (sampled) searches with the oracle."""
    ctx = qis.Context(K=K, R=R, precision=precision, max_n=n, max_instances=n_inst)
    data = []
    for k in range(n_inst):
        J, h = I.instance(ens, n, seed=seed, inst=k)
        phi = I.random_states(n, R, seed=seed + 1000, inst=k)
        iid = ctx.create_instance(J, h)
        ctx.init_states(iid, phi)
        data.append((J, h, phi))
    pairs = [(k, r) for k in range(n_inst) for r in range(R)]
    if sample is not None:
        rng = np.random.default_rng(seed)
        pairs = [pairs[i] for i in sorted(rng.choice(len(pairs), size=min(sample, len(pairs)), replace=False))]
    if per_iter:
        for t in range(1, I_ + 1):
            ctx.iterate(1)
            for k, r in pairs:
                J, h, phi = data[k]
                assert_list_equal(ctx.search_list(k, r), O.qi_search(J, h, K, t, phi[r]), f"t={t} inst={k} r={r}")
    else:
        ctx.iterate(I_)
        for k, r in pairs:
            J, h, phi = data[k]
            assert_list_equal(ctx.search_list(k, r), O.qi_search(J, h, K, I_, phi[r]), f"inst={k} r={r}")
    return ctx, data


@pytest.mark.parametrize("precision", ["fp64", "split_bf16"])
def test_gaussian_n16_every_iteration(precision):
    """N=16 Gaussian, seed 0, K=8, R=4, I=K; merged list vs oracle and 2^16 brute force."""
    n, K, R = 16, 8, 4
    ctx, data = run_pair("gaussian", n, K, R, K, precision, seed=0, per_iter=True)
    J, h, phi = data[0]
    ref = O.qi_multi_search(J, h, K, K, phi)
    got = ctx.topk_states(0, K + 1)
    assert got["count"] == ref["count"]
    assert np.array_equal(got["bits"], ref["bits"])
    assert np.array_equal(got["src"], ref["src"])
    np.testing.assert_allclose(got["E"], ref["E"], rtol=1e-9, atol=0)
    psi, E = O.brute_force(J, h, 1)
    assert int(got["bits"][0, 0]) == int(psi[0]) and got["E"][0] == pytest.approx(E[0], rel=1e-12)


@pytest.mark.parametrize("precision,ens", [("fp64", "gaussian"), ("split_bf16", "gaussian"),
                                           ("split_bf16", "uniform"), ("pm1_fp8", "pm1"), ("fp64", "pm1")])
@pytest.mark.parametrize("n", [70, 130])
def test_ragged_multiword_every_iteration(precision, ens, n):
    """n spans several 64-site tiles and words with a ragged tail; per-iteration parity."""
    run_pair(ens, n, K=20, R=3, I_=12, precision=precision, seed=n, per_iter=True)


@pytest.mark.parametrize("precision,ens", [("split_bf16", "gaussian"), ("pm1_fp8", "pm1")])
def test_many_instances_and_merge(precision, ens):
    n, K, R, I_ = 90, 30, 6, 25
    ctx, data = run_pair(ens, n, K, R, I_, precision, seed=7, n_inst=5)
    for k in range(5):
        J, h, phi = data[k]
        ref = O.qi_multi_search(J, h, K, I_, phi)
        got = ctx.topk_states(k, K + 1)
        assert got["count"] == ref["count"]
        assert np.array_equal(got["bits"], ref["bits"])
        assert np.array_equal(got["src"], ref["src"])
        np.testing.assert_allclose(got["E"], ref["E"], rtol=1e-9)


def test_gaussian_n100_120x32_fp64_sampled():
    """120 instances, N=100, K=120, R=32, FP64; sampled searches vs the oracle."""
    run_pair("gaussian", 100, K=120, R=32, I_=120, precision="fp64", seed=2, n_inst=120, sample=12)


def test_mixed_sizes_one_batch():
    """One context holding instances of different n (the mixed batch of N in {200,350,500,700}),
    scaled down in K and I."""
    ns = [200, 350, 500, 700]
    K, R, I_ = 40, 4, 30
    ctx = qis.Context(K=K, R=R, precision="pm1_fp8", max_n=max(ns), max_instances=len(ns))
    data = []
    for k, n in enumerate(ns):
        J, h = I.instance("pm1", n, seed=44, inst=k)
        phi = I.random_states(n, R, seed=45, inst=k)
        ctx.create_instance(J, h)
        ctx.init_states(k, phi)
        data.append((J, h, phi))
    ctx.iterate(I_)
    for k, (J, h, phi) in enumerate(data):
        for r in (0, R - 1):
            assert_list_equal(ctx.search_list(k, r), O.qi_search(J, h, K, I_, phi[r]), f"n={ns[k]} r={r}")


@pytest.mark.parametrize("precision,ens", [("fp64", "gaussian"), ("split_bf16", "gaussian"), ("pm1_fp8", "pm1")])
def test_full_spectrum_and_exhaustion(precision, ens):
    """K+1 = 2^n: the searches end with the whole sorted spectrum and become inactive."""
    n = 8
    K = 2 ** n - 1
    ctx, data = run_pair(ens, n, K, R=2, I_=2 ** n, precision=precision, seed=9)
    assert ctx.iterate(1, count_active=True) == 0


@pytest.mark.parametrize("precision", ["fp64", "split_bf16"])
def test_small_edge_cases(precision):
    # n = 2 (K < 4), K = 1 (two slots), I = 0
    for n, K, I_ in [(2, 1, 3), (2, 3, 4), (3, 1, 5), (5, 2, 0)]:
        run_pair("gaussian", n, K, R=2, I_=I_, precision=precision, seed=n + K)


def test_library_rng_matches_generator_definition():
    n, R, seed = 77, 5, 1234
    ctx = qis.Context(K=4, R=R, precision="split_bf16", max_n=n, max_instances=2, seed=seed)
    for k in range(2):
        J, h = I.instance("gaussian", n, seed=1, inst=k)
        ctx.create_instance(J, h)
        ctx.init_states(k, None)
        for r in range(R):
            lst = ctx.search_list(k, r)
            assert np.array_equal(lst["bits"][0], I.random_states(n, R, seed=seed, inst=k)[r])


def test_energies_entry_point():
    n = 150
    J, h = I.instance("gaussian", n, seed=5)
    ctx = qis.Context(K=4, R=1, precision="fp64", max_n=n)
    iid = ctx.create_instance(J, h)
    st = I.random_states(n, 50, seed=6)
    np.testing.assert_allclose(ctx.energies(iid, st), O.energies(J, h, st), rtol=1e-12)


def test_invalid_instances_are_rejected():
    n = 10
    ctx = qis.Context(K=4, R=1, precision="split_bf16", max_n=n, max_instances=4)
    J, h = I.instance("gaussian", n, seed=1)
    bad = J.copy(); bad[0, 1] += 1e-3
    with pytest.raises(qis.QISError, match="symmetric"):
        ctx.create_instance(bad, h)
    bad = J.copy(); bad[2, 2] = 1.0
    with pytest.raises(qis.QISError, match="diagonal"):
        ctx.create_instance(bad, h)
    bad = J.copy(); bad[3, 4] = bad[4, 3] = np.nan
    with pytest.raises(qis.QISError, match="NaN"):
        ctx.create_instance(bad, h)
    with pytest.raises(qis.QISError):
        qis.Context(K=4, R=1, precision="pm1_fp8", max_n=n).create_instance(J, h)   # not integer
    iid = ctx.create_instance(J, h)
    assert iid == 0
    with pytest.raises(qis.QISError) as e:
        ctx.iterate(1)                                   # init_states missing
    assert e.value.name == "STATE"


def test_clear_instances_reuses_buffers():
    n, K, R = 40, 10, 2
    ctx = qis.Context(K=K, R=R, precision="split_bf16", max_n=n, max_instances=1)
    for seed in (1, 2):
        ctx.clear_instances()
        J, h = I.instance("gaussian", n, seed=seed)
        phi = I.random_states(n, R, seed=seed)
        ctx.create_instance(J, h)
        ctx.init_states(0, phi)
        ctx.iterate(8)
        assert_list_equal(ctx.search_list(0, 1), O.qi_search(J, h, K, 8, phi[1]))


def test_non_grid_inputs_are_rounded_and_flagged():
    """Inputs finer than the exact grid are rounded onto it (split mode) and reported;
    results then follow the rounded instance, within 1e-9 of the FP64 oracle's energies."""
    n, K, R = 60, 20, 2
    rng = np.random.default_rng(3)
    A = rng.standard_normal((n, n))
    J = np.triu(A, 1) + np.triu(A, 1).T
    h = rng.standard_normal(n)
    ctx = qis.Context(K=K, R=R, precision="split_bf16", max_n=n)
    ctx.create_instance(J, h)
    q, digits, rounded = ctx.instance_info(0)
    assert rounded and q > 30
    phi = I.random_states(n, R, seed=3)
    ctx.init_states(0, phi)
    ctx.iterate(10)
    got = ctx.search_list(0, 0)
    ref = O.qi_search(J, h, K, 10, phi[0])
    assert np.array_equal(got["bits"], ref["bits"][: ref["count"]])
    np.testing.assert_allclose(got["E"], ref["E"][: ref["count"]], rtol=1e-9)


@pytest.mark.parametrize("ens,prec,n,R", [("gaussian", "split_bf16", 100, 4), ("gaussian", "split_bf16", 600, 64),
                                          ("pm1", "pm1_fp8", 1024, 128), ("gaussian", "split_bf16", 200, 20),
                                          ("uniform", "split_bf16", 333, 48)])
def test_tensor_core_fields_equal_exact_simt_fields(monkeypatch, ens, prec, n, R):
    """The tcgen05 digit GEMM and the int64 SIMT reference give bit-identical searches."""
    K, I_ = 30, 6
    J, h = I.instance(ens, n, seed=n, inst=1)
    phi = I.random_states(n, R, seed=n + 1)
    lists = []
    for simt in ("1", "0"):
        monkeypatch.setenv("QIS_FIELDS_SIMT", simt)
        ctx = qis.Context(K=K, R=R, precision=prec, max_n=n)
        ctx.create_instance(J, h)
        ctx.init_states(0, phi)
        ctx.iterate(I_)
        lists.append([ctx.search_list(0, r) for r in range(R)])
        ctx.close()
    for a, b in zip(*lists):
        assert_list_equal(a, b)
