"""The allocation-free entry point, qis_select_candidates_noalloc, against the regular path.

Some callers cannot allocate device memory at the moment they need this work: code running
while a stream is captured into a CUDA graph, real-time loops that must not block in the
driver's allocator, plugins whose device memory belongs to another framework's pool. They call
the allocation-free entry point with their own device buffers. Its output must equal what the
library's regular FP64 path keeps after one iteration from the same parent: the k lowest
(E', c) single and pair flips, with identical FP64 energies.
"""
import numpy as np
import pytest

from paper_2010_00180_gb300 import build, inputs as I, qis

pytestmark = pytest.mark.gpu


def regular_path(J, h, phi, k):
    """k lowest candidates from qis_iterate(1) on a one-search FP64 context."""
    n = h.shape[0]
    ctx = qis.Context(K=k, R=1, precision="fp64", max_n=n)
    ctx.create_instance(J, h)
    ctx.init_states(0, phi[None, :])
    E0 = ctx.search_list(0, 0)["E"][0]
    ctx.iterate(1)
    lst = ctx.search_list(0, 0)
    ctx.close()
    cand = lst["stamp"] != 0          # stamp 0 marks the initial state
    E = lst["E"][cand][:k]
    c = (lst["stamp"][cand] & np.uint64(0xFFFFFFFF)).astype(np.uint32)[:k]
    return E, c, E0


# (n, k, seed): two ordinary calls in a row, then the documented limits (n = 512 fills 2052 of
# a block's 4096 candidate slots, k = 128 the final merge's 8192), a tiny n where k is every
# candidate (n(n+1)/2 = 15) and most blocks hold only padding, and n a multiple of 64 (the
# last word of the state full)
CASES = [(300, 100, 11), (150, 64, 12), (512, 128, 13), (5, 15, 14), (128, 50, 15)]


def test_noalloc_selection_equals_regular_path_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    build.build()
    qis.load()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    for call, (n, k, seed) in enumerate(CASES):
        J, h = I.instance("gaussian", n, seed=seed)
        phi = I.random_states(n, 1, seed=seed + 1)[0]
        dJ = torch.tensor(J, dtype=torch.float64, device=dev)
        dh = torch.tensor(h, dtype=torch.float64, device=dev)
        dbits = torch.tensor(phi.view(np.int64), dtype=torch.int64, device=dev)
        dE = torch.empty(k, dtype=torch.float64, device=dev)
        dc = torch.empty(k, dtype=torch.int32, device=dev)
        dEp = torch.empty(1, dtype=torch.float64, device=dev)
        qis.select_candidates_noalloc(n, dJ.data_ptr(), dh.data_ptr(), dbits.data_ptr(), k, dE.data_ptr(),
                                      dc.data_ptr(), dEp.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize(dev)
        E_ref, c_ref, E0 = regular_path(J, h, phi, k)
        got_E = dE.cpu().numpy()
        got_c = dc.cpu().numpy().view(np.uint32)
        assert np.array_equal(got_E, E_ref), f"call {call}"
        assert np.array_equal(got_c, c_ref), f"call {call}"
        assert dEp.item() == E0


def test_noalloc_rejects_sizes_beyond_its_static_scratch():
    build.build()
    qis.load()
    with pytest.raises(qis.QISError) as e:
        qis.select_candidates_noalloc(513, 1, 1, 1, 8, 1, 1)
    assert e.value.name == "INVALID_ARG" and "512" in str(e.value)
    with pytest.raises(qis.QISError) as e:
        qis.select_candidates_noalloc(100, 1, 1, 1, 129, 1, 1)
    assert e.value.name == "INVALID_ARG"
