"""The request server (include/slm_server.h) on a GPU.

A request's result must not depend on the company it keeps: every graph's
final partition, community count and modularity through the server, with
requests running side by side on several slots, equal those of a run of the
same graph alone (slm_run), and those equal the CPU oracle's.  Admission
respects the HBM budget, and the device memory a run holds stays below the
footprint the server reserved for it.
"""
import time

import numpy as np
import pytest

import graphgen as gg
import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1702_04645_gb300 as slm  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def lib():
    slm.build()
    return slm.load()


def mixed_requests():
    """Graphs of uneven sizes and shapes, each with its own seed and p."""
    out = []
    for k, n in enumerate([1000, 1500, 2400, 3800, 6000, 9500, 15000, 24000]):
        out.append((gg.served_graph(n, 4000 + k), 11 + k, slm.P_HALF if k % 2 else slm.P_ALWAYS))
    out.append((gg.sbm_planted(n_blocks=10, block_size=60, p_in=0.2, p_out=0.01, seed=9), 3, slm.P_HALF))
    out.append((gg.ring_of_cliques(30, 5), 4, slm.P_HALF))
    out.append((gg.star(3000, w=2), 5, slm.P_HALF))
    out.append((gg.isolated_and_loops(40), 6, slm.P_HALF))
    return out


REQS = mixed_requests()


def alone(g, seed, p):
    G = slm.Graph(g.row_ptr, g.col, g.w)
    G.run(seed=seed, accept_p32=p)
    lab, K = G.partition(-1)
    q = G.modularity(-1)
    G.close()
    return lab, K, q


@pytest.fixture(scope="module")
def solo():
    return [alone(g, sd, p) for g, sd, p in REQS]


def test_alone_matches_oracle(solo):
    for (g, sd, p), (lab, K, q) in zip(REQS[:4], solo[:4]):
        r = O.slm(g, seed=sd, P=p)
        assert np.array_equal(lab, r.final)
        assert q == O.modularity(g, r.final)


@pytest.mark.parametrize("slots", [1, 4])
def test_mix_equals_alone(solo, slots):
    sv = slm.Server(budget_bytes=8 << 30, slots=slots)
    tickets = [sv.submit(g.row_ptr, g.col, g.w, seed=sd, accept_p32=p) for g, sd, p in REQS]
    for t in tickets:
        assert sv.wait(t, timeout=120.0)
    infos = [sv.info(t) for t in tickets]
    for t, (lab0, K0, q0), inf in zip(tickets, solo, infos):
        assert inf.state == slm.REQ_DONE
        assert inf.t_submit <= inf.t_admit <= inf.t_done
        assert 0 < inf.peak_bytes <= inf.footprint
        lab, K, q = sv.result(t)
        assert K == K0 and q == q0
        assert np.array_equal(lab, lab0)
    st = sv.stats()
    assert st.completed == len(REQS) and st.failed == 0 and st.queued == 0
    assert st.max_running <= slots
    if slots > 1:
        assert st.max_running > 1, "requests never overlapped"
    sv.close()


def test_budget_limits_concurrency(solo):
    # a budget that holds the largest request once but no two of them
    big = max(slm.footprint(g.n, g.nnz) for g, _, _ in REQS)
    sv = slm.Server(budget_bytes=big + big // 2, slots=4)
    tickets = [sv.submit(g.row_ptr, g.col, g.w, seed=sd, accept_p32=p) for g, sd, p in REQS]
    for t in tickets:
        assert sv.wait(t, timeout=120.0)
    st = sv.stats()
    assert st.max_reserved_bytes <= big + big // 2
    for t, (lab0, K0, q0) in zip(tickets, solo):
        lab, K, q = sv.result(t)
        assert K == K0 and q == q0 and np.array_equal(lab, lab0)
    sv.close()


def test_never_admissible_and_failed_requests():
    sv = slm.Server(budget_bytes=slm.footprint(100, 100), slots=2)
    g = gg.served_graph(5000, 7)
    with pytest.raises(slm.SlmError) as e:
        sv.submit(g.row_ptr, g.col, g.w)
    assert e.value.name == "SLM_ERR_BUDGET"
    assert sv.stats().rejected == 1
    sv.close()

    sv = slm.Server(budget_bytes=1 << 30, slots=2)
    # W_01 = 1 but W_10 missing: validation fails at admission
    bad = sv.submit(np.array([0, 1, 1], np.int32), np.array([1], np.int32))
    good_g = gg.two_cliques(5)
    good = sv.submit(good_g.row_ptr, good_g.col, good_g.w, seed=2)
    assert sv.wait(bad, 60.0) and sv.wait(good, 60.0)
    assert sv.poll(bad) == slm.REQ_FAILED
    with pytest.raises(slm.SlmError) as e:
        sv.result(bad)
    assert e.value.name == "SLM_ERR_NOT_SYMMETRIC"
    lab, K, q = sv.result(good)
    r = O.slm(good_g, seed=2, P=O.P_HALF)
    assert np.array_equal(lab, r.final) and K == 2
    st = sv.stats()
    assert st.failed == 1 and st.completed == 1
    sv.close()


def test_arrivals_while_running(solo):
    """Requests submitted while others run are admitted without waiting for
    the earlier ones to finish, and their results are unchanged."""
    sv = slm.Server(budget_bytes=8 << 30, slots=3)
    order = [7, 0, 1, 6, 2, 3]  # a large request first, small ones arriving behind it
    tickets = []
    for k in order:
        g, sd, p = REQS[k]
        tickets.append(sv.submit(g.row_ptr, g.col, g.w, seed=sd, accept_p32=p))
        time.sleep(0.002)
    for t in tickets:
        assert sv.wait(t, timeout=120.0)
    first = sv.info(tickets[0])
    later = [sv.info(t) for t in tickets[1:]]
    # at least one later request started before the first one ended
    assert any(inf.t_admit < first.t_done for inf in later)
    for t, k in zip(tickets, order):
        lab, K, q = sv.result(t)
        lab0, K0, q0 = solo[k]
        assert K == K0 and q == q0 and np.array_equal(lab, lab0)
    sv.close()


# --------------------------------------------------------------------------
# Cancellation, deadlines and injected allocation failures (all on the host:
# a request stops between sweeps; nothing in flight on the GPU is abandoned)
# --------------------------------------------------------------------------
def _long_graph():
    # the LFR-style recipe does not settle: with a 1,000-sweep limit a run
    # lasts long enough to be caught while it runs
    return gg.lfr_style(n=16384)[0]


def _until(sv, t, state, limit=60.0):
    t0 = time.time()
    while sv.poll(t) != state:
        assert time.time() - t0 < limit, "state never reached"
        time.sleep(0.001)


def test_cancel_running_and_queued_requests(solo):
    sv = slm.Server(budget_bytes=8 << 30, slots=1)
    lg = _long_graph()
    a = sv.submit(lg.row_ptr, lg.col, lg.w, seed=1, max_sweeps=1000)
    g, sd, p = REQS[2]
    b = sv.submit(g.row_ptr, g.col, g.w, seed=sd, accept_p32=p)     # queued behind a
    _until(sv, a, slm.REQ_RUNNING)
    sv.cancel(b)                                                     # queued: ends at once
    assert sv.poll(b) == slm.REQ_FAILED
    ib = sv.info(b)
    assert ib.status == 10 and ib.t_admit == 0.0 and ib.slot == -1
    sv.cancel(a)                                                     # running: next sweep
    assert sv.wait(a, timeout=60.0)
    ia = sv.info(a)
    assert ia.state == slm.REQ_FAILED and ia.status == 10
    with pytest.raises(slm.SlmError) as e:
        sv.result(a)
    assert e.value.name == "SLM_ERR_CANCELLED"
    # the server goes on; a later request's result is unchanged
    c = sv.submit(g.row_ptr, g.col, g.w, seed=sd, accept_p32=p)
    assert sv.wait(c, timeout=60.0)
    lab, K, q = sv.result(c, release=False)
    lab0, K0, q0 = solo[2]
    assert K == K0 and q == q0 and np.array_equal(lab, lab0)
    sv.cancel(c)                                                     # ended: no change
    assert sv.poll(c) == slm.REQ_DONE
    sv.result(c)                                                     # released now
    with pytest.raises(slm.SlmError) as e:
        sv.cancel(c)
    assert e.value.name == "SLM_ERR_INVALID_ARGUMENT"
    st = sv.stats()
    assert st.failed == 2 and st.completed == 1 and st.reserved_bytes == 0
    sv.close()


def test_deadlines_queued_and_running(solo):
    sv = slm.Server(budget_bytes=8 << 30, slots=1)
    lg = _long_graph()
    a = sv.submit(lg.row_ptr, lg.col, lg.w, seed=1, max_sweeps=1000, deadline=0.4)
    g, sd, p = REQS[1]
    b = sv.submit(g.row_ptr, g.col, g.w, seed=sd, accept_p32=p, deadline=0.05)
    c = sv.submit(g.row_ptr, g.col, g.w, seed=sd, accept_p32=p, deadline=600.0)
    assert sv.wait(b, timeout=60.0)
    ib = sv.info(b)
    assert ib.state == slm.REQ_FAILED and ib.status == 11 and ib.t_admit == 0.0
    assert sv.wait(a, timeout=60.0)
    ia = sv.info(a)
    assert ia.state == slm.REQ_FAILED and ia.status == 11
    assert ia.t_admit > 0 and ia.t_done - ia.t_submit >= 0.4
    assert sv.wait(c, timeout=60.0)
    lab, K, q = sv.result(c)
    lab0, K0, q0 = solo[1]
    assert K == K0 and q == q0 and np.array_equal(lab, lab0)
    with pytest.raises(slm.SlmError):
        sv.submit(g.row_ptr, g.col, g.w, deadline=-1.0)
    assert sv.stats().reserved_bytes == 0
    sv.close()


def test_injected_allocation_failure_fails_one_request(solo):
    sv = slm.Server(budget_bytes=8 << 30, slots=1)
    g, sd, p = REQS[0]
    slm.debug_fail_allocation(5)
    try:
        t = sv.submit(g.row_ptr, g.col, g.w, seed=sd, accept_p32=p)
        assert sv.wait(t, timeout=60.0)
    finally:
        slm.debug_fail_allocation(0)
    inf = sv.info(t)
    assert inf.state == slm.REQ_FAILED and inf.status == 4
    t2 = sv.submit(g.row_ptr, g.col, g.w, seed=sd, accept_p32=p)
    assert sv.wait(t2, timeout=60.0)
    lab, K, q = sv.result(t2)
    lab0, K0, q0 = solo[0]
    assert K == K0 and q == q0 and np.array_equal(lab, lab0)
    assert sv.stats().reserved_bytes == 0
    sv.close()


def test_destroy_while_threads_wait():
    """Threads blocked in wait() when the server is destroyed return once
    their request has ended; destroy frees nothing they still use."""
    import threading
    sv = slm.Server(budget_bytes=8 << 30, slots=1)
    lg = _long_graph()
    ts = [sv.submit(lg.row_ptr, lg.col, lg.w, seed=1, max_sweeps=40) for _ in range(3)]
    done = []
    h = sv._h.value
    lib = slm.load()

    def waiter(t):
        done.append(lib.slm_server_wait(h, t, -1.0))

    th = [threading.Thread(target=waiter, args=(t,)) for t in ts]
    for x in th:
        x.start()
    _until(sv, ts[0], slm.REQ_RUNNING)
    time.sleep(0.2)   # every waiter is inside wait() before destroy begins
    sv.close()
    for x in th:
        x.join(timeout=120.0)
        assert not x.is_alive()
    assert sorted(done) == [0, 0, 0]


def test_directed_requests_equal_directed_runs():
    """Directed requests (slm_server_submit_directed: W as out-arcs, the
    directed Q_w) mixed with undirected ones on four slots: each equals the
    same graph run alone, which equals the directed oracle."""
    dig = [gg.random_directed(300 + 90 * k, 0.03, 70 + k, wmax=4, loops=0.1, recip=0.3)
           for k in range(4)]
    dig.append(gg.lfr_directed(5000, 0.5, 0.4)[0])
    solo_d = []
    for k, g in enumerate(dig):
        G = slm.Graph(g.row_ptr, g.col, g.w, directed=True)
        G.run(seed=20 + k, accept_p32=slm.P_HALF)
        solo_d.append((G.partition(-1), G.modularity(-1)))
        G.close()
    r = O.directed_slm(dig[0], seed=20, P=O.P_HALF)
    assert np.array_equal(solo_d[0][0][0], r.final)
    sv = slm.Server(budget_bytes=8 << 30, slots=4)
    td = [sv.submit(g.row_ptr, g.col, g.w, seed=20 + k, accept_p32=slm.P_HALF, directed=True)
          for k, g in enumerate(dig)]
    tu = [sv.submit(g.row_ptr, g.col, g.w, seed=sd, accept_p32=p) for g, sd, p in REQS[:4]]
    for t in td + tu:
        assert sv.wait(t, timeout=120.0)
    # a directed request is costed for U = W + W^T and its packed strengths
    g = dig[-1]
    assert sv.info(td[-1]).footprint == slm.load().slm_server_footprint(g.n, 2 * g.nnz) + 8 * (g.n + 1)
    for t, ((lab0, K0), q0) in zip(td, solo_d):
        assert sv.info(t).state == slm.REQ_DONE
        lab, K, q = sv.result(t)
        assert K == K0 and q == q0 and np.array_equal(lab, lab0)
    sv.close()
