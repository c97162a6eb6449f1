"""Pins of the oracle's directed restatement of the method (the ord_* functions:
Q_w with out- and in-strengths, Section 2.4).

Every directed value is checked against the directed modularity numerator
evaluated by brute force (a double sum over node pairs), against networkx's
directed modularity, by exhaustive search, and by reduction: on a symmetric W
the directed method must reproduce the symmetric oracle's every decision, each
value being exactly twice the symmetric one.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle as O
from brute import (brute_max_q_num_directed, components, dense, q_num_def_directed, tail)


def digraphs():
    out = []
    for seed in range(14):
        n = 5 + seed % 8
        out.append(gg.random_directed(n, 0.3, seed, wmax=5, loops=0.3 if seed % 2 else 0.0,
                                      recip=0.4 if seed % 3 else 0.0))
    # a directed cycle, a directed star in and out, a tournament-like dense graph
    out.append(gg.directed_from_edges(7, np.arange(7), (np.arange(7) + 1) % 7))
    out.append(gg.directed_from_edges(6, np.zeros(5, np.int64), np.arange(1, 6)))
    out.append(gg.directed_from_edges(6, np.arange(1, 6), np.zeros(5, np.int64)))
    out.append(gg.random_directed(9, 0.6, 99, wmax=2, recip=0.5))
    return out


def tie_digraphs():
    """Unit weights: many exactly equal scores."""
    return [gg.random_directed(8 + s % 4, 0.35, 600 + s, wmax=1, recip=0.5) for s in range(10)]


def sym_graphs():
    out = [gg.random_small(6 + s % 7, 0.45, s, wmax=5, loops=0.3 if s % 2 else 0.0)
           for s in range(10)]
    return out + [gg.two_cliques(4), gg.path(9), gg.star(6), gg.ring_of_cliques(4, 3),
                  gg.isolated_and_loops(7)]


def _unbrs(g):
    """U-neighbours of every node (out- and in-neighbours, itself excluded)."""
    W = dense(g)
    U = W + W.T
    return [[int(j) for j in np.flatnonzero(U[i]) if j != i] for i in range(g.n)]


def _state(g, seed):
    a = O.directed_assign(g)
    nb = _unbrs(g)
    rng = np.random.default_rng(seed)
    for _ in range(3):
        i = int(rng.integers(0, g.n))
        if nb[i]:
            a[i] = nb[i][int(rng.integers(0, len(nb[i])))]
    return a, O.rootlabel(a)


def _random_state(g, seed):
    nb = _unbrs(g)
    rng = np.random.default_rng(seed)
    a = np.arange(g.n, dtype=np.int32)
    for i in range(g.n):
        if nb[i]:
            a[i] = nb[i][int(rng.integers(0, len(nb[i])))]
    return a, O.rootlabel(a)


def states():
    out = [(g, _state(g, gi)) for gi, g in enumerate(digraphs())]
    out += [(g, _random_state(g, 50 + gi)) for gi, g in enumerate(digraphs() + tie_digraphs())]
    out += [(g, (np.arange(g.n, dtype=np.int32), np.arange(g.n, dtype=np.int32)))
            for g in tie_digraphs()]
    return out


# --------------------------------------------------------------------------
# directed modularity: definition, networkx, special cases
# --------------------------------------------------------------------------
def test_directed_modularity_matches_definition_and_networkx():
    nx = pytest.importorskip("networkx")
    from networkx.algorithms.community import modularity as nxmod
    rng = np.random.default_rng(3)
    for gi, g in enumerate(digraphs()):
        W = dense(g)
        for k in (1, 2, 3, g.n):
            lab = rng.integers(0, k, g.n).astype(np.int32)
            assert O.directed_modularity_num(g, lab) == q_num_def_directed(W, lab)
            D = nx.DiGraph()
            D.add_nodes_from(range(g.n))
            for u in range(g.n):
                for p in range(g.row_ptr[u], g.row_ptr[u + 1]):
                    D.add_edge(u, int(g.col[p]), weight=int(g.w[p]))
            comms = [set(np.flatnonzero(lab == c).tolist()) for c in np.unique(lab)]
            assert abs(O.directed_modularity(g, lab) - nxmod(D, comms, weight="weight")) < 1e-12
    g = digraphs()[0]
    assert O.directed_modularity_num(g, np.zeros(g.n, np.int32)) == 0  # one community
    empty = gg.directed_from_edges(4, [], [])
    assert O.directed_modularity(empty, np.arange(4)) == 0.0


def test_directed_strengths_and_symmetrise():
    for g in digraphs():
        W = dense(g)
        so, si, m = O.directed_strengths(g)
        assert (so == W.sum(1)).all() and (si == W.sum(0)).all() and m == W.sum()
        u = O.symmetrise(g)
        assert (dense(u) == W + W.T).all()
        for i in range(u.n):
            c = u.col[u.row_ptr[i]:u.row_ptr[i + 1]]
            assert (np.diff(c) > 0).all()


# --------------------------------------------------------------------------
# symmetric input: the directed method is the symmetric one, values doubled
# --------------------------------------------------------------------------
def test_directed_on_symmetric_graphs_reduces_to_symmetric_oracle():
    for gi, g in enumerate(sym_graphs()):
        assert (O.directed_assign(g) == O.assign(g)).all()
        a = O.assign(g)
        rng = np.random.default_rng(gi)
        for _ in range(2):
            i = int(rng.integers(0, g.n))
            nb = [int(j) for j in g.col[g.row_ptr[i]:g.row_ptr[i + 1]] if j != i]
            if nb:
                a[i] = nb[int(rng.integers(0, len(nb)))]
        root = O.rootlabel(a)
        b1, ga1, g1 = O.scan(g, root)
        b2, ga2, g2 = O.directed_scan(g, root)
        assert (b1 == b2).all() and (ga2 == 2 * ga1).all() and (g2 == 2 * g1).all()
        for i in np.flatnonzero(ga1 > 0):
            assert O.directed_branch_gain(g, a, root, int(i), int(b1[i])) == \
                2 * O.branch_gain(g, a, root, int(i), int(b1[i]))
            assert O.directed_target(g, root, int(i), int(b1[i])) == \
                O.target(g, root, int(i), int(b1[i]))
        pa, pr, pk = O.positive(g, a)
        da, dr, dk = O.directed_positive(g, a)
        assert (pa == da).all() and (pr == dr).all() and pk == dk
        assert O.directed_modularity_num(g, root) == O.modularity_num(g, root)


@pytest.mark.parametrize("P", [O.P_HALF, O.P_ALWAYS])
def test_directed_run_on_symmetric_graphs_equals_symmetric_run(P):
    graphs = sym_graphs() + [gg.sbm_planted(n_blocks=4, block_size=30, p_in=0.3, p_out=0.03,
                                            seed=5), gg.random_small(80, 0.08, 41, loops=0.1)]
    for g in graphs:
        r1 = O.slm(g, seed=7, P=P)
        r2 = O.directed_slm(g, seed=7, P=P)
        assert r1.num_levels == r2.num_levels and r1.top == r2.top
        for (l1, k1), (l2, k2) in zip(r1.levels, r2.levels):
            assert k1 == k2 and (l1 == l2).all()
        assert r1.stats == r2.stats and (r1.trace == r2.trace).all()
        assert (r1.final == r2.final).all()


# --------------------------------------------------------------------------
# every directed value against the directed numerator
# --------------------------------------------------------------------------
def test_directed_assign_brute_force():
    for g in digraphs() + tie_digraphs():
        W = dense(g)
        a = O.directed_assign(g)
        single = np.arange(g.n)
        q0 = q_num_def_directed(W, single)
        for i in range(g.n):
            d = {}
            for j in _unbrs(g)[i]:
                lab = single.copy()
                lab[i] = j
                d[j] = q_num_def_directed(W, lab) - q0
            if not d or max(d.values()) <= 0:
                assert a[i] == i
            else:
                top = max(d.values())
                assert a[i] == min(j for j in d if d[j] == top)


def test_directed_scan_gain_identity_and_argmax():
    for g, (a, root) in states():
        W = dense(g)
        best, gain, gl = O.directed_scan(g, root)
        q0 = q_num_def_directed(W, root)
        for i in range(g.n):
            ci = int(root[i])
            # leaving to a fresh singleton changes the numerator by -g(i)
            lab = root.astype(np.int64).copy()
            lab[i] = g.n + 1
            assert q_num_def_directed(W, lab) - q0 == -gl[i]
            d = {}
            for j in _unbrs(g)[i]:
                C = int(root[j])
                if C == ci or C in d:
                    continue
                lab = root.astype(np.int64).copy()
                lab[i] = C
                d[C] = q_num_def_directed(W, lab) - q0
            if d and max(d.values()) > 0:
                top = max(d.values())
                assert best[i] == min(C for C in d if d[C] == top) and gain[i] == top
            else:
                assert best[i] == ci and gain[i] == 0


def test_directed_branch_gain_identity():
    checked = 0
    for g, (a, root) in states():
        W = dense(g)
        best, gain, _ = O.directed_scan(g, root)
        q0 = q_num_def_directed(W, root)
        for i in np.flatnonzero(gain > 0):
            B = int(best[i])
            S = tail(a, int(i))
            lab = root.astype(np.int64).copy()
            lab[S] = B
            assert O.directed_branch_gain(g, a, root, int(i), B) == q_num_def_directed(W, lab) - q0
            checked += 1
    assert checked > 40


def test_directed_target_brute_force():
    for g, (a, root) in states():
        W = dense(g)
        single = np.arange(g.n)
        q0 = q_num_def_directed(W, single)
        for i in range(g.n):
            for B in {int(root[j]) for j in _unbrs(g)[i]} - {int(root[i])}:
                sc = {}
                for j in _unbrs(g)[i]:
                    if root[j] != B:
                        continue
                    lab = single.copy()
                    lab[i] = j
                    sc[j] = q_num_def_directed(W, lab) - q0  # the pair score
                top = max(sc.values())
                assert O.directed_target(g, root, i, B) == min(j for j in sc if sc[j] == top)


def _split_options(a, root, A):
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
        if u not in cyc:
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


def _directed_positive_by_definition(g, a):
    """POSITIVE with the local gains and every split measured on the directed
    numerator."""
    W = dense(g)
    a = a.copy()
    while True:
        root = components(a)
        q0 = q_num_def_directed(W, root)
        flagged = None
        for A in sorted(set(root.tolist())):
            for i in np.flatnonzero(root == A):
                lab = root.copy()
                lab[i] = g.n + 1
                if q_num_def_directed(W, lab) - q0 > 0:  # leaving raises Q: g(i) < 0
                    flagged = A
                    break
            if flagged is not None:
                break
        if flagged is None:
            return a
        best = None
        for ty, u, v, b in _split_options(a, root, flagged):
            d = q_num_def_directed(W, components(b)) - q0
            key = (-d, ty, u, v)
            if best is None or key < best[0]:
                best = (key, b)
        a = best[1]


def test_directed_positive_matches_definition_level_search():
    nsplit = 0
    for g, (a, _) in states():
        a2, root2, k = O.directed_positive(g, a)
        nsplit += k
        assert (a2 == _directed_positive_by_definition(g, a)).all()
        assert (root2 == components(a2)).all()
        _, _, gl = O.directed_scan(g, root2)
        assert (gl >= 0).all()
    assert nsplit > 5


# --------------------------------------------------------------------------
# AGGREGATE keeps a directed graph directed
# --------------------------------------------------------------------------
def test_directed_aggregate_invariants():
    for gi, g in enumerate(digraphs()):
        a, root = _state(g, 300 + gi)
        idv, K = O.compact(root)
        h = O.aggregate(g, idv, K)
        W = dense(g)
        Pm = np.zeros((g.n, K), np.int64)
        Pm[np.arange(g.n), idv] = 1
        assert (dense(h) == Pm.T @ W @ Pm).all()
        so, si, m = O.directed_strengths(g)
        so2, si2, m2 = O.directed_strengths(h)
        assert m2 == m
        assert (so2 == np.bincount(idv, weights=so, minlength=K)).all()
        assert (si2 == np.bincount(idv, weights=si, minlength=K)).all()
        assert O.directed_modularity_num(h, np.arange(K)) == O.directed_modularity_num(g, idv)


# --------------------------------------------------------------------------
# whole runs: exhaustive bound, determinism, stop condition
# --------------------------------------------------------------------------
@pytest.mark.parametrize("P", [O.P_HALF, O.P_ALWAYS])
def test_directed_run_vs_exhaustive(P):
    for g in [d for d in digraphs() if d.n <= 9]:
        W = dense(g)
        best_num, _ = brute_max_q_num_directed(W)
        r = O.directed_slm(g, seed=11, P=P)
        num = O.directed_modularity_num(g, r.final)
        assert num == q_num_def_directed(W, r.final)
        assert num <= best_num
        assert num >= q_num_def_directed(W, np.arange(g.n))  # never below singletons
        r2 = O.directed_slm(g, seed=11, P=P)
        assert (r2.final == r.final).all() and r.stats == r2.stats


def test_directed_run_degenerate_graphs():
    for n in (0, 1, 5):
        g = gg.directed_from_edges(n, [], [])
        r = O.directed_slm(g)
        assert r.num_levels == 0 and (r.final == np.arange(n)).all()
    loops = gg.directed_from_edges(4, np.arange(4), np.arange(4), [1, 2, 3, 4])
    r = O.directed_slm(loops)
    assert r.num_levels == 0
    with pytest.raises(ValueError):
        O.directed_slm(gg.directed_from_edges(2, [0], [1], [1 << 30]))


def test_directed_orientation_changes_decisions():
    """The directed null model is not the symmetric one on W + W^T: a node
    whose arcs all leave it is scored by s_out * Sigma_in, so some digraph
    must make a different choice than the symmetric method on U."""
    differ = 0
    for g in digraphs() + tie_digraphs():
        u = O.symmetrise(g)
        differ += int((O.directed_assign(g) != O.assign(u)).any())
    assert differ > 0
