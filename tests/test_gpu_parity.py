"""Parity of the CUDA path with the CPU oracle, element by element.

Every step of the method is run through the C ABI (``include/slm_steps.h``)
on the same seeded inputs as the oracle and compared exactly: all the
arithmetic is integer, so the bar is bit-exact, and the one FP64 quotient
(modularity) is computed by the same expression on both sides.
"""
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


def small_graphs():
    out = [
        ("two_cliques5", gg.two_cliques(5)),
        ("ring30x5", gg.ring_of_cliques(30, 5)),
        ("path300", gg.path(300)),
        ("star300", gg.star(300)),
        ("star5000", gg.star(5000, w=3)),
        ("isolated", gg.isolated_and_loops(50)),
        ("single", gg.from_edges(1, [], [])),
        ("sbm8x100", gg.sbm_planted(n_blocks=8, block_size=100, p_in=0.1, p_out=0.005, seed=4)),
        ("rmat12", gg.rmat(scale=12, seed=5)),
        ("forest3000", gg.forest_sbm_graph(3000, 12, 77)),
        ("ties", gg.random_small(300, 0.03, 11, wmax=1)),
    ]
    for k in range(6):
        out.append((f"rand{k}", gg.random_small(40 + 17 * k, 0.12, 100 + k, wmax=6,
                                                loops=0.3 if k % 2 else 0.0)))
    return out


GRAPHS = small_graphs()
IDS = [n for n, _ in GRAPHS]


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.int32)).cuda()


def host(t, n=None):
    a = t.cpu().numpy()
    return a if n is None else a[:n]


def states(g, seed):
    """Assignment graphs to test on: ASSIGN's, ASSIGN's with random re-pointings,
    and every node pointing at a random neighbour (long cycles)."""
    rng = np.random.default_rng(seed)
    a0 = O.assign(g)
    a1 = a0.copy()
    for _ in range(max(3, g.n // 10)):
        i = int(rng.integers(0, max(g.n, 1)))
        nb = g.col[g.row_ptr[i]:g.row_ptr[i + 1]]
        if g.n and nb.shape[0]:
            a1[i] = nb[int(rng.integers(0, nb.shape[0]))]
    a2 = np.arange(g.n, dtype=np.int32)
    for i in range(g.n):
        nb = [int(j) for j in g.col[g.row_ptr[i]:g.row_ptr[i + 1]] if j != i]
        if nb:
            a2[i] = nb[int(rng.integers(0, len(nb)))]
    return [a0, a1, a2]


# --------------------------------------------------------------------------
# single steps
# --------------------------------------------------------------------------
@pytest.mark.parametrize("name,g", GRAPHS, ids=IDS)
def test_strengths_and_assign(name, g):
    s, m = slm.step_strengths(g.row_ptr, g.col, g.w)
    so, mo = O.strengths(g)
    assert m == mo
    assert (host(s, g.n) == so).all()
    a = slm.step_assign(g.row_ptr, g.col, g.w, s, m)
    assert (host(a, g.n) == O.assign(g)).all()


def test_components_random_functional_graphs():
    rng = np.random.default_rng(1)
    cases = [np.arange(1, dtype=np.int32), np.array([1, 0], np.int32)]
    for n in (2, 7, 33, 1000, 4097, 70000):
        cases.append(rng.integers(0, n, size=n).astype(np.int32))
        p = rng.permutation(n).astype(np.int32)          # one permutation: cycles only
        cases.append(p)
        chain = np.arange(n, dtype=np.int32) - 1          # a deep chain into a 1-cycle
        chain[0] = 0
        cases.append(chain)
        big = np.roll(np.arange(n, dtype=np.int32), -1)   # one long cycle
        cases.append(big)
    for a in cases:
        root = slm.step_components(a)
        assert (host(root, a.shape[0]) == O.rootlabel(a)).all()


@pytest.mark.parametrize("name,g", GRAPHS, ids=IDS)
def test_scan(name, g):
    s, m = O.strengths(g)
    for k, a in enumerate(states(g, 1)):
        root = O.rootlabel(a)
        best, gain, gl = slm.step_scan(g.row_ptr, g.col, g.w, s.astype(np.int32), m, root)
        ob, og, ogl = O.scan(g, root)
        assert (host(best, g.n) == ob).all(), (name, k)
        assert (host(gain, g.n) == og).all(), (name, k)
        assert (host(gl, g.n) == ogl).all(), (name, k)


@pytest.mark.parametrize("name,g", GRAPHS, ids=IDS)
def test_branch_gain(name, g):
    s, m = O.strengths(g)
    for k, a in enumerate(states(g, 2)):
        root = O.rootlabel(a)
        ob, og, _ = O.scan(g, root)
        bg = host(slm.step_branch_gain(g.row_ptr, g.col, g.w, s.astype(np.int32), m, a, root,
                                       ob, torch.from_numpy(og)), g.n)
        cand = np.flatnonzero(og > 0)
        if cand.shape[0] > 300:
            cand = np.random.default_rng(k).choice(cand, 300, replace=False)
        for i in cand:
            assert bg[i] == O.branch_gain(g, a, root, int(i), int(ob[i])), (name, k, int(i))
        assert (bg[og <= 0] == 0).all()


def oracle_maximal(g, a, seed, P, level, sweep):
    """One synchronous MAXIMAL with the oracle's step functions."""
    s, m = O.strengths(g)
    root = O.rootlabel(a)
    best, gain, _ = O.scan(g, root)
    acc = []
    npos = 0
    for i in np.flatnonzero(gain > 0):
        if O.branch_gain(g, a, root, int(i), int(best[i])) > 0:
            npos += 1
            if O.draw(seed, level, sweep, int(i)) < P:
                acc.append(int(i))
    new = a.copy()
    for i in acc:
        new[i] = O.target(g, root, i, int(best[i]))
    return new, (int((gain > 0).sum()), npos, len(acc))


@pytest.mark.parametrize("name,g", [x for x in GRAPHS if x[1].n <= 3000],
                         ids=[n for n, x in GRAPHS if x.n <= 3000])
def test_maximal_step(name, g):
    s, m = O.strengths(g)
    for k, a in enumerate(states(g, 3)):
        a, _, _ = O.positive(g, a)
        root = O.rootlabel(a)
        for P in (O.P_HALF, O.P_ALWAYS):
            na, cnt = slm.step_maximal(g.row_ptr, g.col, g.w, s.astype(np.int32), m, a, root,
                                       seed=7, accept_p32=P, level=1, sweep=k)
            ra, rc = oracle_maximal(g, a, 7, P, 1, k)
            assert tuple(int(x) for x in cnt) == rc, (name, k)
            assert (host(na, g.n) == ra).all(), (name, k)


@pytest.mark.parametrize("name,g", GRAPHS, ids=IDS)
def test_positive(name, g):
    s, m = O.strengths(g)
    for k, a in enumerate(states(g, 4)):
        na, nroot, splits = slm.step_positive(g.row_ptr, g.col, g.w, s.astype(np.int32), m, a)
        oa, oroot, osplits = O.positive(g, a)
        assert splits == osplits, (name, k)
        assert (host(na, g.n) == oa).all(), (name, k)
        assert (host(nroot, g.n) == oroot).all(), (name, k)


@pytest.mark.parametrize("name,g", GRAPHS, ids=IDS)
def test_compact_aggregate_modularity(name, g):
    for k, a in enumerate(states(g, 5)):
        root = O.rootlabel(a)
        idv, K = slm.step_compact(root)
        oid, oK = O.compact(root)
        assert K == oK
        assert (host(idv, g.n) == oid).all()
        rp2, col2, w2 = slm.step_aggregate(g.row_ptr, g.col, g.w, oid, oK)
        h = O.aggregate(g, oid, oK)
        assert (host(rp2, oK + 1) == h.row_ptr).all()
        assert (host(col2) == h.col).all() and (host(w2) == h.w).all()
        q, num = slm.step_modularity(g.row_ptr, g.col, g.w, oid)
        assert num == O.modularity_num(g, oid)
        assert q == O.modularity(g, oid)          # same expression, bit-equal


# --------------------------------------------------------------------------
# whole runs (Algorithm 1)
# --------------------------------------------------------------------------
def compare_run(g, seed, P, flags=0, max_sweeps=1000):
    G = slm.Graph(g.row_ptr, g.col, g.w)
    G.run(seed=seed, accept_p32=P, max_sweeps=max_sweeps, flags=flags)
    r = O.slm(g, seed=seed, P=P, max_sweeps=max_sweeps, flags=flags)
    tr = G.trace()
    assert tr.shape == r.trace.shape and (tr == r.trace).all(), "per-sweep trace differs"
    assert G.num_levels() == r.num_levels
    for l, (ids, K) in enumerate(r.levels):
        lab, k = G.partition(l)
        assert k == K and (lab == ids).all(), f"level {l} differs"
        st = G.stats(l)
        assert (st.sweeps, st.status, st.moves, st.splits, st.candidates, st.edges_scanned) == r.stats[l]
        assert G.modularity(l) == O.modularity(g, _compose(r, l, g.n))
    fin, k = G.partition(-1)
    assert (fin == r.final).all()
    assert G.modularity(-1) == O.modularity(g, r.final)
    return G, r


def _compose(r, l, n):
    lab = np.arange(n, dtype=np.int32)
    for t in range(l + 1):
        lab = r.levels[t][0][lab]
    return lab


@pytest.mark.parametrize("name,g", GRAPHS, ids=IDS)
@pytest.mark.parametrize("P", [O.P_HALF, O.P_ALWAYS], ids=["p_half", "p_one"])
def test_full_run(name, g, P):
    compare_run(g, seed=3, P=P)


def test_full_run_no_positive_and_sweep_limit():
    g = gg.rmat(scale=11, seed=9)
    compare_run(g, seed=1, P=O.P_HALF, flags=O.FLAG_NO_POSITIVE)
    compare_run(g, seed=1, P=O.P_HALF, max_sweeps=3)


def test_sbm_planted_config_full_run():
    """The 10,000-node planted partition (20 blocks of 500, intra/inter degree 16/4)."""
    g = gg.sbm_planted()
    G, r = compare_run(g, seed=1, P=O.P_HALF)
    assert G.modularity(-1) > 0.7


@pytest.mark.parametrize("mu_t,mu_w", [(0.2, 0.1), (0.5, 0.4), (0.8, 0.7)])
def test_weighted_lfr_mixing_pairs_full_run(mu_t, mu_w):
    """The paper's benchmark family at its three mixing pairs (10,000 nodes,
    mean degree 50): every level, sweep and the final partition as the oracle's."""
    g, _ = gg.lfr_weighted(10000, mu_t, mu_w)
    compare_run(g, seed=1, P=O.P_HALF)


def test_invalid_inputs_are_rejected():
    g = gg.random_small(20, 0.3, 1)
    bad = g.w.copy()
    bad[0] += 1                     # W no longer symmetric
    with pytest.raises(slm.SlmError) as e:
        slm.Graph(g.row_ptr, g.col, bad)
    assert e.value.status == 2
    col = g.col.copy()
    col[1], col[0] = col[0], col[1]  # unsorted row
    with pytest.raises(slm.SlmError) as e:
        slm.Graph(g.row_ptr, col, g.w)
    assert e.value.status == 1
    neg = g.w.copy()
    neg[:] = -1
    with pytest.raises(slm.SlmError):
        slm.Graph(g.row_ptr, g.col, neg)
    big = np.full_like(g.w, 2**28)  # m_w >= 2^31
    with pytest.raises(slm.SlmError) as e:
        slm.Graph(g.row_ptr, g.col, big)
    assert e.value.status == 3
    G = slm.Graph(g.row_ptr, g.col, g.w)
    with pytest.raises(slm.SlmError) as e:
        G.num_levels()
    assert e.value.status == 6


def test_invalid_entries_in_long_rows_are_rejected():
    """The validator spreads a row over many warps: a defect anywhere in a hub
    row (at a warp boundary, deep inside, in its last entry) is still found."""
    rng = np.random.default_rng(5)
    n = 6000
    leaves = np.arange(1, n)
    u = np.concatenate([np.zeros(n - 1, np.int64), rng.integers(1, n, 3000)])
    v = np.concatenate([leaves, rng.integers(1, n, 3000)])
    g = gg.from_edges(n, u, v, rng.integers(1, 5, u.shape[0]))
    slm.Graph(g.row_ptr, g.col, g.w).close()  # valid
    lo, hi = int(g.row_ptr[0]), int(g.row_ptr[1])
    assert hi - lo > 4000
    for p in (lo + 32, lo + 2049, hi - 1):
        bad = g.w.copy()
        bad[p] += 1  # W_0j != W_j0
        with pytest.raises(slm.SlmError) as e:
            slm.Graph(g.row_ptr, g.col, bad)
        assert e.value.status == 2, p
    for p in (lo + 64, lo + 3001):
        col = g.col.copy()
        col[p], col[p - 1] = col[p - 1], col[p]  # unsorted across a warp boundary
        with pytest.raises(slm.SlmError) as e:
            slm.Graph(g.row_ptr, col, g.w)
        assert e.value.status == 1, p
    col = g.col.copy()
    col[hi - 1] = n  # out of range in the row's last entry
    with pytest.raises(slm.SlmError) as e:
        slm.Graph(g.row_ptr, col, g.w)
    assert e.value.status == 1


def test_scan_tuning_changes_no_result():
    """Every launch shape of the scan gives the same outputs (the autotuner
    relies on it), and the autotuner returns a valid tuning."""
    from paper_1702_04645_gb300 import tune
    g = gg.rmat(scale=14, seed=9)
    rp, col, w = dev(g.row_ptr), dev(g.col), dev(g.w)
    s, m = slm.step_strengths(rp, col, w)
    a = slm.step_assign(rp, col, w, s, m)
    a, root, _ = slm.step_positive(rp, col, w, s, m, a)
    start = slm.get_scan_tuning()
    ref = [host(t) for t in slm.step_scan(rp, col, w, s, m, root)]
    try:
        for t in ({"streams": 1}, {"blocks_large": 1, "blocks_mid": 2, "blocks_warp": 4},
                  {"blocks_group": 32, "blocks_hub": 16, "blocks_small": 4},
                  {"shape_alt": 0x7FF}, {"shape_alt": 0x555}, {"shape_alt": 0x2AA, "streams": 1}):
            slm.set_scan_tuning(**t)
            out = [host(x) for x in slm.step_scan(rp, col, w, s, m, root)]
            for x, y in zip(out, ref):
                assert np.array_equal(x, y)
        best, rep = tune.autotune_scan(g.row_ptr, g.col, g.w, reps=2, use_cache=False)
        assert set(best) == set(start)
        assert rep["best_ms"] <= rep["start_ms"]
    finally:
        slm.set_scan_tuning(**start)
    with pytest.raises(slm.SlmError):
        slm.set_scan_tuning(streams=3)
    assert slm.get_scan_tuning() == start


@pytest.mark.parametrize("shape_alt", [0x7FF, 0x555, 0x2AA])
def test_scan_alternative_shapes_equal_oracle(shape_alt):
    """Each fine degree class's second launch shape gives the oracle's scan:
    rows of every class from 1 to 4096 entries (the stars add a 3,000-entry
    row) and, beside them, hub rows."""
    start = slm.get_scan_tuning()
    try:
        slm.set_scan_tuning(shape_alt=shape_alt)
        for g in (gg.rmat(scale=13, seed=4), gg.star(3000, w=2), gg.star(1500),
                  gg.sbm_planted(n_blocks=8, block_size=100, p_in=0.1, p_out=0.005, seed=4)):
            s, m = O.strengths(g)
            for k, a in enumerate(states(g, 3)):
                root = O.rootlabel(a)
                best, gain, gl = slm.step_scan(g.row_ptr, g.col, g.w, s.astype(np.int32), m, root)
                ob, og, ol = O.scan(g, root)
                assert (host(best, g.n) == ob).all() and (host(gain, g.n) == og).all()
                assert (host(gl, g.n) == ol).all()
    finally:
        slm.set_scan_tuning(**start)
