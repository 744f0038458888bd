"""Failure detection on the GPU without a GPU fault.

Both failures are made on purpose in the allowed forms: a survivor buffer that is too small
for the candidates an instance produces (every candidate of the all-zero Hamiltonian ties),
and a device-side wait on a barrier that nothing completes (the library's wait probe) with a
short bound. Each must come back as an error code from the next synchronising call, with no
hang and no fault, and the context must stay usable: after qis_clear_instances or qis_reset
the searches equal the oracle again."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2010_00180_gb300 import build, inputs as I, qis

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    qis.load()


def same_as_oracle(ctx, iid, J, h, K, iters, phi, R):
    for r in range(R):
        got = ctx.search_list(iid, r)
        ref = O.qi_search(J, h, K, iters, phi[r])
        c = ref["count"]
        assert got["count"] == c
        assert np.array_equal(got["bits"], ref["bits"][:c]) and np.array_equal(got["E"], ref["E"][:c])
        assert np.array_equal(got["stamp"], ref["stamp"][:c]) and np.array_equal(got["used"], ref["used"][:c])


def test_survivor_overflow_is_reported_and_the_context_recovers():
    """All-zero J and h: every single and pair flip has dE = 0, so all n(n+1)/2 = 2080
    candidates of n = 64 survive the first iteration's filter, far above survivor_cap = 72
    (the smallest allowed for K = 1). The filters write at most cap entries; the merge sees the
    count and raises the capacity flag instead of reading past the buffer."""
    n, K, R = 64, 1, 2
    ctx = qis.Context(K=K, R=R, precision="split_bf16", max_n=n, max_instances=1, survivor_cap=4 * (K + 1) + 64)
    ctx.create_instance(np.zeros((n, n)), np.zeros(n))
    ctx.init_states(0, I.random_states(n, R, seed=5))
    ctx.iterate(1)
    with pytest.raises(qis.QISError) as e:
        ctx.synchronize()
    assert e.value.name == "CAPACITY"
    with pytest.raises(qis.QISError) as e:        # reported until the searches are restarted
        ctx.iterate(1, count_active=True)
    assert e.value.name == "CAPACITY"
    # recovery: a new instance in the same context runs exactly as the oracle
    ctx.clear_instances()
    J, h = I.instance("gaussian", n, seed=6)
    phi = I.random_states(n, R, seed=7)
    ctx.create_instance(J, h)
    ctx.init_states(0, phi)
    ctx.iterate(6)
    ctx.synchronize()
    same_as_oracle(ctx, 0, J, h, K, 6, phi, R)
    ctx.close()


@pytest.mark.parametrize("prec,ens", [("split_bf16", "gaussian"), ("pm1_fp8", "pm1")])
def test_device_wait_timeout_is_reported_and_the_context_recovers(prec, ens):
    """The field GEMM's MMA thread waits on a barrier nothing completes, bounded by 1 ms: the
    wait runs out, the kernel drains the copies it issued, frees its tensor memory and returns;
    the next synchronising call reports DEVICE_TIMEOUT. With the probe off and the default
    bound, qis_reset restarts the searches and they equal the oracle."""
    n, K, R, iters = 200, 20, 8, 7
    J, h = I.instance(ens, n, seed=8)
    phi = I.random_states(n, R, seed=9)
    ctx = qis.Context(K=K, R=R, precision=prec, max_n=n, max_instances=1)
    ctx.create_instance(J, h)
    ctx.init_states(0, phi)
    ctx.set_wait_limit(1_000_000, probe=True)
    ctx.iterate(1)                 # the first iteration computes every parent's fields on the GEMM
    with pytest.raises(qis.QISError) as e:
        ctx.synchronize()
    assert e.value.name == "DEVICE_TIMEOUT"
    ctx.set_wait_limit(2_000_000_000, probe=False)
    ctx.reset()
    ctx.iterate(iters)
    ctx.synchronize()
    same_as_oracle(ctx, 0, J, h, K, iters, phi, R)
    ctx.close()


def test_wait_limit_arguments_are_checked():
    ctx = qis.Context(K=4, R=1, precision="split_bf16", max_n=16)
    for limit, probe in [(10, 0), (10 ** 12, 0), (10 ** 9, 2)]:
        with pytest.raises(qis.QISError) as e:
            ctx.set_wait_limit(limit, probe)
        assert e.value.name == "INVALID_ARG"
    ctx.close()
