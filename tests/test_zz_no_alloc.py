"""The modularity entry point that allocates no device memory.

Callers that cannot let a library call cudaMalloc (frameworks that have
handed all device memory to their own caching allocator or arena) use
slm_step_modularity_noalloc, whose scratch is one fixed device array.  Its
results must equal those of slm_step_modularity, which allocates its scratch
per call, on consecutive calls that reuse the shared array.
"""
import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1702_04645_gb300 as slm  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def lib():
    slm.build()
    return slm.load()


def labelled(g, seed, k):
    rng = np.random.default_rng(seed)
    return rng.integers(0, max(1, min(k, g.n)), size=g.n).astype(np.int32)


def test_noalloc_equals_allocating_entry_point_on_consecutive_calls():
    big = gg.rmat(scale=14, seed=3)
    small = gg.random_small(60, 0.2, 4, wmax=5, loops=0.3)
    cases = [(big, labelled(big, 1, 300)), (small, labelled(small, 2, 7)),
             (big, np.arange(big.n, dtype=np.int32)), (small, np.zeros(small.n, np.int32))]
    for g, lab in cases:  # each call reuses the scratch the previous one left behind
        q_ref, num_ref = slm.step_modularity(g.row_ptr, g.col, g.w, lab)
        q, num = slm.step_modularity_noalloc(g.row_ptr, g.col, g.w, lab)
        assert num == num_ref          # exact integer numerator
        assert q == q_ref              # same FP64 expression: bit-equal


def test_noalloc_rejects_oversized_and_out_of_range_inputs():
    n = (1 << 20) + 1
    rp = np.zeros(n + 1, np.int32)
    with pytest.raises(slm.SlmError) as e:
        slm.step_modularity_noalloc(rp, np.zeros(1, np.int32), np.ones(1, np.int32),
                                    np.zeros(n, np.int32))
    assert e.value.status == 1
    g = gg.random_small(30, 0.3, 5)
    bad = np.zeros(g.n, np.int32)
    bad[3] = g.n + 5
    with pytest.raises(slm.SlmError) as e:
        slm.step_modularity_noalloc(g.row_ptr, g.col, g.w, bad)
    assert e.value.status == 1
    # the shared scratch still gives the right answer afterwards
    lab = labelled(g, 9, 4)
    assert slm.step_modularity_noalloc(g.row_ptr, g.col, g.w, lab) == \
        slm.step_modularity(g.row_ptr, g.col, g.w, lab)


def test_noalloc_call_leaves_device_memory_unchanged():
    """The defining property: with every input and output already on the
    device, a call changes neither the device's free memory nor what the
    caching allocator holds (nothing is allocated, not even temporarily
    from a pool that would keep the memory afterwards)."""
    import ctypes as C
    g = gg.rmat(scale=14, seed=7)
    lab = labelled(g, 3, 200)
    dev = [torch.as_tensor(np.ascontiguousarray(x, dtype=np.int32)).cuda()
           for x in (g.row_ptr, g.col, g.w, lab)]
    num = torch.zeros(1, dtype=torch.int64, device="cuda")
    q = torch.zeros(1, dtype=torch.float64, device="cuda")
    lib = slm.load()

    def call():
        st = lib.slm_step_modularity_noalloc(g.n, *(C.c_void_p(t.data_ptr()) for t in dev),
                                             C.c_void_p(num.data_ptr()), C.c_void_p(q.data_ptr()),
                                             C.c_void_p(0))
        assert st == 0
    call()  # the first call on the device looks up the array's address
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(3):
        call()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_reserved() == reserved0
    q_ref, num_ref = slm.step_modularity(g.row_ptr, g.col, g.w, lab)
    assert int(num.item()) == num_ref and float(q.item()) == q_ref
