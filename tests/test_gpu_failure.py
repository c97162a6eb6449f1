"""Failure detection on the GPU without a GPU fault.

The cooperative kernels (all rounds of POSITIVE in one launch) meet at grid
barriers whose waits have a time limit.  Here a block is made to leave before
the first barrier, so that the others' waits run out: the launch must end,
report SLM_ERR_TIMEOUT through the C ABI, and leave the context usable for a
normal run whose result still equals the oracle's.
"""
import ctypes as C

import numpy as np
import pytest

import graphgen as gg
import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1702_04645_gb300 as slm  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    slm.build()
    return slm.load()


def test_barrier_passes_when_every_block_arrives(lib):
    for blocks in (1, 2, 16, 152):
        assert lib.slm_check_grid_barrier(blocks, -1, 1.0, None) == 0


def test_barrier_wait_runs_out_and_context_survives(lib):
    # block 1 never arrives: the other blocks give up after 50 ms
    assert lib.slm_check_grid_barrier(8, 1, 0.05, None) == 8
    assert b"ran out of time" in lib.slm_last_error(None)
    # the context is still usable: a full run matches the oracle
    g = gg.sbm_planted(n_blocks=6, block_size=60, p_in=0.2, p_out=0.01, seed=21)
    G = slm.Graph(g.row_ptr, g.col, g.w)
    G.run(seed=3, accept_p32=slm.P_HALF)
    lab, _ = G.partition(-1)
    r = O.slm(g, seed=3, P=O.P_HALF)
    assert np.array_equal(lab, r.final)
    torch.cuda.synchronize()


def test_barrier_rejects_non_resident_grids(lib):
    assert lib.slm_check_grid_barrier(0, -1, 1.0, None) == 1
    assert lib.slm_check_grid_barrier(10 ** 6, -1, 1.0, None) == 1
    assert lib.slm_check_grid_barrier(4, 4, 1.0, None) == 1


# --------------------------------------------------------------------------
# Allocation failures, injected on the host (slm_debug_fail_allocation): the
# k-th device allocation is refused before the CUDA call is made.
# --------------------------------------------------------------------------
def _graph():
    return gg.sbm_planted(n_blocks=8, block_size=70, p_in=0.2, p_out=0.01, seed=31)


def test_injected_allocation_failure_in_create(lib):
    g = _graph()
    failed = 0
    try:
        for k in range(1, 12):
            slm.debug_fail_allocation(k)
            try:
                G = slm.Graph(g.row_ptr, g.col, g.w)
            except slm.SlmError as e:
                assert e.status == 4, e          # SLM_ERR_OUT_OF_MEMORY
                assert b"injected" in lib.slm_last_error(None)
                failed += 1
                continue
            finally:
                slm.debug_fail_allocation(0)
            G.close()
    finally:
        slm.debug_fail_allocation(0)
    assert failed >= 4                            # the copies of row_ptr, col, w and s
    G = slm.Graph(g.row_ptr, g.col, g.w)
    G.run(seed=2, accept_p32=slm.P_HALF)
    assert np.array_equal(G.partition(-1)[0], O.slm(g, seed=2, P=O.P_HALF).final)
    G.close()


def test_injected_allocation_failure_in_run_keeps_previous_results(lib):
    g = _graph()
    r = O.slm(g, seed=4, P=O.P_HALF)
    G = slm.Graph(g.row_ptr, g.col, g.w)
    # a handle whose first run fails has no results
    slm.debug_fail_allocation(1)
    with pytest.raises(slm.SlmError) as ex:
        G.run(seed=4, accept_p32=slm.P_HALF)
    slm.debug_fail_allocation(0)
    assert ex.value.status == 4
    with pytest.raises(slm.SlmError) as ex:
        G.partition(-1)
    assert ex.value.status == 6                   # SLM_ERR_NOT_RUN
    G.run(seed=4, accept_p32=slm.P_HALF)
    ref, K = G.partition(-1)
    q = G.modularity(-1)
    assert np.array_equal(ref, r.final)
    failed = 0
    for k in list(range(1, 40)) + [60, 100, 200, 400]:
        slm.debug_fail_allocation(k)
        try:
            G.run(seed=4, accept_p32=slm.P_HALF)
            ok = True
        except slm.SlmError as e:
            assert e.status == 4, e
            ok = False
            failed += 1
        finally:
            slm.debug_fail_allocation(0)
        lab, K2 = G.partition(-1)               # the previous (or the new) run's results
        assert np.array_equal(lab, ref) and K2 == K and G.modularity(-1) == q
        assert G.num_levels() == r.num_levels
        if ok:
            break
    assert failed >= 10
    G.run(seed=4, accept_p32=slm.P_HALF)
    assert np.array_equal(G.partition(-1)[0], ref)
    G.close()
    torch.cuda.synchronize()
