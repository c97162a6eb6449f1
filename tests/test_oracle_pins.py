"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks one oracle function against something other than itself:
a library routine, the definition evaluated by brute force, a closed form, an
exhaustive search, or an invariant.  Graphs are tiny so the suite stays fast.
"""
import os

import numpy as np
import pytest

import graphgen as gg
import oracle as O
from brute import (brute_max_q_num, components, dense, q_num_def, set_partitions, tail)

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def small_graphs():
    out = []
    for seed in range(12):
        n = 5 + seed % 9
        out.append(gg.random_small(n, 0.45, seed, wmax=5, loops=0.3 if seed % 2 else 0.0))
    out += [gg.two_cliques(4), gg.path(9), gg.star(6), gg.ring_of_cliques(4, 3),
            gg.isolated_and_loops(7)]
    return out


def random_labels(n, seed, k):
    rng = np.random.default_rng(seed)
    return rng.integers(0, max(k, 1), size=n).astype(np.int32)


# --------------------------------------------------------------------------
# splitmix64: published reference outputs
# --------------------------------------------------------------------------
def test_mix64_matches_published_sequence():
    gold = [l.split() for l in open(os.path.join(GOLD, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    G = 0x9E3779B97F4A7C15
    for k, val in gold:
        assert O.mix64((int(k) * G) % 2**64) == int(val, 16)


def test_draw_is_uniformish_and_keyed():
    d = [O.draw(7, 0, 0, i) for i in range(4000)]
    assert 0.45 < np.mean(np.array(d) < 2**31) < 0.55
    assert O.draw(7, 0, 0, 5) != O.draw(7, 0, 1, 5) != O.draw(7, 1, 0, 5)
    assert O.draw(7, 0, 0, 5) != O.draw(8, 0, 0, 5)


# --------------------------------------------------------------------------
# modularity (Section 2.4)
# --------------------------------------------------------------------------
def test_modularity_matches_definition_double_sum():
    for gi, g in enumerate(small_graphs()):
        W = dense(g)
        for k in (1, 2, 3, g.n):
            lab = random_labels(g.n, gi * 10 + k, k)
            assert O.modularity_num(g, lab) == q_num_def(W, lab)


def test_modularity_matches_networkx_directed():
    nx = pytest.importorskip("networkx")
    from networkx.algorithms.community import modularity as nxmod
    for gi, g in enumerate(small_graphs()):
        if g.nnz == 0:
            continue
        D = nx.DiGraph()
        D.add_nodes_from(range(g.n))
        for u in range(g.n):
            for p in range(g.row_ptr[u], g.row_ptr[u + 1]):
                D.add_edge(u, int(g.col[p]), weight=int(g.w[p]))
        lab = random_labels(g.n, gi, 3)
        comms = [set(np.flatnonzero(lab == c).tolist()) for c in np.unique(lab)]
        assert abs(O.modularity(g, lab) - nxmod(D, comms, weight="weight")) < 1e-12


def test_modularity_special_cases():
    for g in small_graphs():
        if g.nnz == 0:
            assert O.modularity(g, np.zeros(g.n, np.int32)) == 0.0
            continue
        # one community: Q = 0 exactly (Section 2.4)
        assert O.modularity_num(g, np.zeros(g.n, np.int32)) == 0
        # singletons: sum_i (m W_ii - s_i^2)
        W = dense(g)
        s = W.sum(1)
        m = int(W.sum())
        assert O.modularity_num(g, np.arange(g.n, dtype=np.int32)) == int(
            (m * np.diag(W) - s * s).sum())
        # undirected bound Q in [-1/2, 1]
        for k in range(4):
            q = O.modularity(g, random_labels(g.n, k, 1 + k))
            assert -0.5 <= q <= 1.0


def test_closed_forms():
    rows = [l.split() for l in open(os.path.join(GOLD, "closed_forms.txt"))
            if l.strip() and not l.startswith("#")]
    for name, k, r, q in rows:
        k, r, q = int(k), int(r), float(q)
        if name == "two_cliques":
            g = gg.two_cliques(k)
            lab = np.repeat([0, 1], k).astype(np.int32)
        elif name == "ring_singles":
            g = gg.ring_of_cliques(r, k)
            lab = np.repeat(np.arange(r), k).astype(np.int32)
        else:
            g = gg.ring_of_cliques(r, k)
            lab = np.repeat(np.arange(r) // 2, k).astype(np.int32)
        assert abs(O.modularity(g, lab) - q) < 1e-15


# --------------------------------------------------------------------------
# ASSIGN (Section 3.1)
# --------------------------------------------------------------------------
def test_assign_brute_force_and_cycle_length():
    assert (O.assign(zero_gain_graph()) == [0, 1, 3, 2]).all()   # zero gain: self-assigned
    for g in small_graphs() + tie_graphs() + [gg.random_small(60, 0.1, 99, wmax=3)]:
        W = dense(g)
        s = W.sum(1)
        m = int(W.sum())
        a = O.assign(g)
        for i in range(g.n):
            # the gain of joining {j} measured on the definition
            base = np.arange(g.n)
            q0 = q_num_def(W, base)
            best, bestj = 0, i
            for j in range(g.n):
                if j == i or W[i, j] == 0:
                    continue
                lab = base.copy()
                lab[i] = j
                d = q_num_def(W, lab) - q0
                if d > best:
                    best, bestj = d, j
            assert a[i] == bestj
        # one out-edge per node; cycles have length <= 2
        for v in range(g.n):
            x = v
            for _ in range(g.n):
                x = a[x]
            assert a[a[x]] == x


# --------------------------------------------------------------------------
# COMPONENTS (Section 3.2)
# --------------------------------------------------------------------------
def test_rootlabel_against_brute_force():
    rng = np.random.default_rng(3)
    for n in (1, 2, 5, 17, 64):
        for _ in range(20):
            a = rng.integers(0, n, size=n).astype(np.int32)
            assert (O.rootlabel(a) == components(a)).all()


def test_rootlabel_components_match_networkx():
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(4)
    a = rng.integers(0, 300, size=300).astype(np.int32)
    root = O.rootlabel(a)
    G = nx.Graph()
    G.add_nodes_from(range(300))
    G.add_edges_from((i, int(a[i])) for i in range(300))
    for comp in nx.connected_components(G):
        assert len({int(root[v]) for v in comp}) == 1
    assert len(set(root.tolist())) == nx.number_connected_components(G)


# --------------------------------------------------------------------------
# MAXIMAL's per-node scan: gain identity and argmax (Section 3.4)
# --------------------------------------------------------------------------
def _state(g, seed):
    """A reachable state: ASSIGN then POSITIVE, plus a few random re-pointings."""
    a = O.assign(g)
    rng = np.random.default_rng(seed)
    for _ in range(3):
        i = int(rng.integers(0, g.n))
        nb = g.col[g.row_ptr[i]:g.row_ptr[i + 1]]
        if nb.shape[0]:
            a[i] = nb[int(rng.integers(0, nb.shape[0]))]
    return a, O.rootlabel(a)


def _random_state(g, seed):
    """Every node points at a random neighbour: assignment graphs with long cycles."""
    rng = np.random.default_rng(seed)
    a = np.arange(g.n, dtype=np.int32)
    for i in range(g.n):
        nb = [int(j) for j in g.col[g.row_ptr[i]:g.row_ptr[i + 1]] if j != i]
        if nb:
            a[i] = nb[int(rng.integers(0, len(nb)))]
    return a, O.rootlabel(a)


def zero_gain_graph():
    """m_w = 16 and s_0 = s_1 = 4, W_01 = 1: joining node 1 gains exactly zero."""
    return gg.from_edges(4, [0, 0, 1, 2], [0, 1, 1, 3], [3, 1, 3, 4])


def tie_graphs():
    """Unit weights and equal degrees: many exactly equal gains."""
    return [zero_gain_graph(), gg.path(7), gg.ring_of_cliques(6, 3), gg.star(5),
            gg.from_edges(8, np.arange(8), (np.arange(8) + 1) % 8)] + [
        gg.random_small(9 + s % 4, 0.4, 500 + s, wmax=1) for s in range(10)]


def test_scan_gain_identity_and_argmax():
    states = [(g, _state(g, gi)) for gi, g in enumerate(small_graphs())]
    states += [(g, _random_state(g, gi)) for gi, g in enumerate(tie_graphs())]
    for g in tie_graphs():   # singletons: every neighbour community ties on degree
        states.append((g, (np.arange(g.n, dtype=np.int32), np.arange(g.n, dtype=np.int32))))
    for g, (a, root) in states:
        W = dense(g)
        best, gain, gl = O.scan(g, root)
        q0 = q_num_def(W, root)
        for i in range(g.n):
            # leaving for a fresh singleton changes Q's numerator by -2 g(i)
            lab = root.copy()
            lab[i] = g.n + 1
            assert q_num_def(W, lab) - q0 == -2 * gl[i]
            # every neighbouring community: the chosen one is the best, smallest name on ties
            cands = {}
            for j in np.flatnonzero(W[i]):
                if j == i or root[j] == root[i]:
                    continue
                lab = root.copy()
                lab[i] = root[j]
                cands[int(root[j])] = q_num_def(W, lab) - q0
            pos = {c: d for c, d in cands.items() if d > 0}
            if not pos:
                assert best[i] == root[i] and gain[i] == 0
            else:
                top = max(pos.values())
                assert best[i] == min(c for c, d in pos.items() if d == top)
                assert 2 * gain[i] == top


# --------------------------------------------------------------------------
# Branch gain and target (Algorithm MAXIMAL)
# --------------------------------------------------------------------------
def test_branch_gain_identity():
    checked = 0
    for gi, g in enumerate(small_graphs() + [gg.random_small(30, 0.2, 5)]):
        W = dense(g)
        a, root = _state(g, 100 + gi)
        q0 = q_num_def(W, root)
        comms = sorted(set(root.tolist()))
        for i in range(g.n):
            S = tail(a, i)
            for B in comms:
                if B == root[i]:
                    continue
                lab = root.copy()
                lab[S] = B
                d = q_num_def(W, lab) - q0
                assert 2 * O.branch_gain(g, a, root, i, B) == d
                checked += 1
    assert checked > 200


def test_target_brute_force():
    states = [(g, _state(g, gi)) for gi, g in enumerate(small_graphs())]
    states += [(g, _random_state(g, gi)) for gi, g in enumerate(tie_graphs())]
    states += [(g, (np.arange(g.n), np.arange(g.n, dtype=np.int32))) for g in tie_graphs()]
    for g, (a, root) in states:
        W = dense(g)
        s = W.sum(1)
        m = int(W.sum())
        for i in range(g.n):
            for B in set(root[np.flatnonzero(W[i])].tolist()) - {int(root[i])}:
                js = [j for j in np.flatnonzero(W[i]) if j != i and root[j] == B]
                sc = {j: m * W[i, j] - s[i] * s[j] for j in js}
                top = max(sc.values())
                assert O.target(g, root, i, B) == min(j for j in js if sc[j] == top)


# --------------------------------------------------------------------------
# POSITIVE (Section 3.3): post-condition and the choice of every split,
# measured on the definition
# --------------------------------------------------------------------------
def _split_options(a, root, A):
    """Every candidate bisection of community A as (type, u, v, new a)."""
    n = len(a)
    mem = [v for v in range(n) if root[v] == A]
    x = mem[0]
    for _ in range(n):
        x = a[x]
    cyc = [x]
    y = a[x]
    while y != x:
        cyc.append(y)
        y = a[y]
    opts = []
    for u in mem:
        if u in cyc:
            continue
        b = a.copy()
        b[u] = u
        opts.append((0, u, -1, b))
    for p in range(len(cyc)):
        for q in range(p + 1, len(cyc)):
            b = a.copy()
            b[cyc[p]] = cyc[p]
            b[cyc[q]] = cyc[q]
            u, v = sorted((cyc[p], cyc[q]))
            opts.append((1, u, v, b))
    return opts


def _positive_by_definition(g, a):
    """POSITIVE with every split scored by recomputing the numerator."""
    W = dense(g)
    s = W.sum(1)
    m = int(W.sum())
    a = a.copy()
    while True:
        root = components(a)
        flagged = None
        for A in sorted(set(root.tolist())):
            mem = np.flatnonzero(root == A)
            sig = s[mem].sum()
            for i in mem:
                k = sum(W[i, j] for j in mem if j != i)
                if m * k - s[i] * (sig - s[i]) < 0:
                    flagged = A
                    break
            if flagged is not None:
                break
        if flagged is None:
            return a
        q0 = q_num_def(W, root)
        best = None
        for ty, u, v, b in _split_options(a, root, flagged):
            d = q_num_def(W, components(b)) - q0
            key = (-d, ty, u, v)
            if best is None or key < best[0]:
                best = (key, b)
        a = best[1]


def test_positive_matches_definition_level_search():
    graphs = small_graphs() + [gg.random_small(14, 0.35, s, wmax=3) for s in range(20, 30)]
    states = [(g, _state(g, 200 + gi)[0]) for gi, g in enumerate(graphs)]
    states += [(g, _random_state(g, 300 + gi)[0]) for gi, g in enumerate(graphs + tie_graphs())]
    # states whose best bisections tie: two branch cuts; branch and cycle cuts
    states.append((gg.random_small(8, 0.5, 7278, wmax=1), np.array([3, 5, 5, 0, 5, 1, 3, 5], np.int32)))
    states.append((gg.random_small(8, 0.5, 7388, wmax=1), np.array([5, 2, 0, 6, 7, 7, 3, 0], np.int32)))
    # two cycle cuts with the same smaller node tie for best
    states.append((gg.random_small(10, 0.6, 16811, wmax=1),
                   np.array([6, 5, 0, 5, 2, 9, 8, 9, 4, 1], np.int32)))
    nsplit = 0
    for g, a in states:
        a2, root2, k = O.positive(g, a)
        nsplit += k
        ref = _positive_by_definition(g, a)
        assert (a2 == ref).all()
        assert (root2 == components(a2)).all()
        # post-condition: no node with a negative local gain
        _, _, gl = O.scan(g, root2)
        assert (gl >= 0).all()
    assert nsplit > 5


# --------------------------------------------------------------------------
# Compaction and AGGREGATE (Section 3.5)
# --------------------------------------------------------------------------
def test_compact_and_aggregate_invariants():
    for gi, g in enumerate(small_graphs() + [gg.random_small(50, 0.1, 77, loops=0.2)]):
        a, root = _state(g, 300 + gi)
        idv, K = O.compact(root)
        names = sorted(set(root.tolist()))
        assert K == len(names)
        assert all(idv[v] == names.index(root[v]) for v in range(g.n))
        h = O.aggregate(g, idv, K)
        W = dense(g)
        P = np.zeros((g.n, K), dtype=np.int64)
        P[np.arange(g.n), idv] = 1
        assert (dense(h) == P.T @ W @ P).all()          # W' = P^T W P
        for r in range(K):                               # sorted unique columns
            c = h.col[h.row_ptr[r]:h.row_ptr[r + 1]]
            assert (np.diff(c) > 0).all()
        s, m = O.strengths(g)
        s2, m2 = O.strengths(h)
        assert m2 == m
        assert (s2 == np.bincount(idv, weights=s, minlength=K).astype(np.int64)).all()
        assert O.modularity_num(h, np.arange(K, dtype=np.int32)) == O.modularity_num(g, idv)


# --------------------------------------------------------------------------
# The whole method (Algorithm 1)
# --------------------------------------------------------------------------
def _final_merge_gains(g, lab):
    W = dense(g)
    s = W.sum(1)
    m = int(W.sum())
    K = int(lab.max()) + 1 if g.n else 0
    P = np.zeros((g.n, K), dtype=np.int64)
    P[np.arange(g.n), lab] = 1
    WA = P.T @ W @ P
    S = P.T @ s
    out = m * WA - np.outer(S, S)
    np.fill_diagonal(out, np.iinfo(np.int64).min)
    out[WA == 0] = np.iinfo(np.int64).min
    return out


@pytest.mark.parametrize("P", [O.P_HALF, O.P_ALWAYS])
def test_run_on_tiny_graphs_vs_exhaustive(P):
    for seed in range(25):
        n = 6 + seed % 5
        g = gg.random_small(n, 0.5, 1000 + seed, wmax=4, loops=0.2 if seed % 3 == 0 else 0)
        r = O.slm(g, seed=seed, P=P)
        W = dense(g)
        best_num, _ = brute_max_q_num(W)
        num = O.modularity_num(g, r.final)
        assert num <= best_num
        assert num == q_num_def(W, r.final)
        # final labels are the composition of the recorded levels
        lab = np.arange(g.n)
        for l, (ids, K) in enumerate(r.levels):
            assert ids.max() + 1 == K
            lab = ids[lab]
        assert (lab == r.final).all()
        # converged top level: no two final communities gain by merging
        if r.top[0] == 0 and g.nnz:
            assert (_final_merge_gains(g, r.final) <= 0).all()


def test_run_two_cliques_closed_form():
    for k in (4, 5):
        g = gg.two_cliques(k)
        for P in (O.P_HALF, O.P_ALWAYS):
            for seed in range(4):
                r = O.slm(g, seed=seed, P=P)
                assert (r.final == np.repeat([0, 1], k)).all()
                best, _ = brute_max_q_num(dense(g))
                assert O.modularity_num(g, r.final) == best
                assert abs(O.modularity(g, r.final) - (k * (k - 1) / (k * (k - 1) + 1) - 0.5)) < 1e-15


def test_run_ring_of_cliques_runs_of_whole_cliques():
    r_, k = 30, 5
    g = gg.ring_of_cliques(r_, k)
    m = r_ * (k * (k - 1) + 2)
    for P in (O.P_HALF, O.P_ALWAYS):
        run = O.slm(g, seed=3, P=P)
        lab = run.final
        clique_lab = lab.reshape(r_, k)
        assert (clique_lab == clique_lab[:, :1]).all()       # whole cliques
        per = clique_lab[:, 0]
        # rotate so that a community boundary sits at index 0, then read runs
        start = next(c for c in range(r_) if per[c] != per[c - 1]) if len(set(per)) > 1 else 0
        rot = np.roll(per, -start)
        runs = []
        cur, ln = rot[0], 0
        for x in rot:
            if x == cur:
                ln += 1
            else:
                runs.append(ln)
                cur, ln = x, 1
        runs.append(ln)
        assert len(runs) == len(set(per))                   # each community is one run
        q = sum((gsz * k * (k - 1) + 2 * (gsz - 1)) / m - (gsz * (k * (k - 1) + 2) / m) ** 2
                for gsz in runs)
        assert abs(O.modularity(g, lab) - q) < 1e-12
        assert O.modularity(g, lab) >= 0.8757575757575757 - 1e-12


def test_run_invariants_and_determinism():
    g = gg.sbm_planted(n_blocks=4, block_size=60, p_in=0.2, p_out=0.01, seed=9)
    r1 = O.slm(g, seed=5)
    r2 = O.slm(g, seed=5)
    assert (r1.final == r2.final).all()
    assert r1.stats == r2.stats
    s, m = O.strengths(g)
    cur = g
    for ids, K in r1.levels:
        st, mt = O.strengths(cur)
        assert mt == m
        assert np.bincount(ids, weights=st, minlength=K).sum() == m
        cur = O.aggregate(cur, ids, K)
    q = O.modularity(g, r1.final)
    assert -0.5 <= q <= 1.0 and q > 0.5


def test_run_degenerate_graphs():
    # empty graph and isolated nodes: singletons, no level, Q = 0
    for g in (gg.from_edges(0, [], []), gg.from_edges(5, [], []), gg.isolated_and_loops(6)):
        r = O.slm(g)
        assert r.num_levels == 0
        assert (r.final == np.arange(g.n)).all()
    # a star is one community
    r = O.slm(gg.star(8))
    assert r.num_levels == 1 and r.levels[0][1] == 1
