"""Pins of the oracle's classical (sequential-move) Louvain, the method the
paper builds on and names for comparison (Section 6).

The oracle's run is compared level by level with a definition-level
restatement that scores every candidate move by recomputing the modularity
numerator, and checked for local optimality, against the exhaustive optimum,
on closed-form graphs and on degenerate inputs.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle as O
from brute import brute_max_q_num, dense, q_num_def


def louvain_by_definition(W):
    """Levels (ids, K) and the final labels of sequential-move Louvain, every
    move measured on the definition's numerator."""
    n0 = W.shape[0]
    final = np.arange(n0)
    levels = []
    Wl = W.copy()
    while True:
        n = Wl.shape[0]
        comm = np.arange(n)
        passes, first = 0, 0
        while True:
            moves = 0
            for i in range(n):
                q0 = q_num_def(Wl, comm)
                best = None
                for C in sorted({int(comm[j]) for j in np.flatnonzero(Wl[i]) if j != i}
                                - {int(comm[i])}):
                    lab = comm.copy()
                    lab[i] = C
                    d = q_num_def(Wl, lab) - q0
                    if d > 0 and (best is None or d > best[0]):
                        best = (d, C)
                if best is not None:
                    comm[i] = best[1]
                    moves += 1
            passes += 1
            if passes == 1:
                first = moves
            if moves == 0:
                break
        names = np.unique(comm)
        K = names.shape[0]
        ids = np.searchsorted(names, comm)
        if first == 0 or K == n:
            return levels, final
        levels.append((ids, K))
        final = ids[final]
        P = np.zeros((n, K), np.int64)
        P[np.arange(n), ids] = 1
        Wl = P.T @ Wl @ P


def graphs():
    out = [gg.random_small(5 + s % 8, 0.45, 700 + s, wmax=5, loops=0.3 if s % 2 else 0.0)
           for s in range(14)]
    out += [gg.random_small(9 + s % 4, 0.4, 800 + s, wmax=1) for s in range(8)]  # ties
    return out + [gg.two_cliques(4), gg.path(9), gg.star(6), gg.ring_of_cliques(4, 3),
                  gg.isolated_and_loops(7)]


def test_louvain_matches_definition_level_run():
    total_levels = 0
    for g in graphs():
        levels, final = louvain_by_definition(dense(g))
        r = O.louvain(g)
        assert r.num_levels == len(levels)
        for (a, ka), (b, kb) in zip(r.levels, levels):
            assert ka == kb and (a == b).all()
        assert (r.final == final).all()
        total_levels += len(levels)
    assert total_levels > 15


def _level_graphs(g, r):
    out = [g]
    for ids, K in r.levels[:-1]:
        out.append(O.aggregate(out[-1], ids, K))
    return out


def test_louvain_levels_are_local_optima():
    """At the end of every level no single node move raises the numerator."""
    for g in [gg.random_small(60, 0.08, 31, loops=0.1), gg.sbm_planted(n_blocks=3, block_size=20,
              p_in=0.4, p_out=0.05, seed=2), gg.random_small(40, 0.15, 33, wmax=1)]:
        r = O.louvain(g)
        assert r.num_levels >= 1
        for h, (ids, K) in zip(_level_graphs(g, r), r.levels):
            W = dense(h)
            q0 = q_num_def(W, ids)
            for i in range(h.n):
                for C in {int(ids[j]) for j in np.flatnonzero(W[i]) if j != i} - {int(ids[i])}:
                    lab = ids.copy()
                    lab[i] = C
                    assert q_num_def(W, lab) - q0 <= 0


def test_louvain_bounded_by_the_exhaustive_optimum():
    for g in [x for x in graphs() if x.n <= 10]:
        W = dense(g)
        best, _ = brute_max_q_num(W)
        r = O.louvain(g)
        num = q_num_def(W, r.final)
        assert num <= best
        assert num >= q_num_def(W, np.arange(g.n))


def test_louvain_closed_forms_and_invariants():
    r = O.louvain(gg.two_cliques(5))
    lab = r.final
    assert len(set(lab[:5])) == 1 and len(set(lab[5:])) == 1 and lab[0] != lab[5]
    g = gg.ring_of_cliques(30, 5)
    r = O.louvain(g)
    # every clique lies inside one community
    assert all(len(set(r.final[5 * c:5 * c + 5].tolist())) == 1 for c in range(30))
    # per level: moves are the trace's moves, entries scanned are passes x entries
    for lv, st in enumerate(r.stats):
        rows = r.trace[r.trace[:, 0] == lv]
        assert st[0] == rows.shape[0] and st[2] == int(rows[:, 4].sum())
    assert r.stats[0][5] == r.stats[0][0] * g.nnz
    r2 = O.louvain(g)
    assert (r2.final == r.final).all()


@pytest.mark.parametrize("n", [0, 1, 5])
def test_louvain_degenerate_graphs(n):
    g = gg.from_edges(n, [], [])
    r = O.louvain(g)
    assert r.num_levels == 0 and (r.final == np.arange(n)).all()
    loops = gg.isolated_and_loops(max(n, 1))
    assert O.louvain(loops).num_levels == 0
