"""Pins of the whole-array recomputations used by the full-size GPU tests
(tests/whole_array.py): on small graphs they must give exactly the pinned
oracle's ASSIGN and MAXIMAL scan (Sections 3.1 and 3.4), for ASSIGN's own
state and for random assignment states; the planted mistakes below (a tie
broken the wrong way, the node's own edge counted, the strict threshold
relaxed) must each be caught by the same comparison."""
import numpy as np
import pytest

import graphgen as gg
import oracle as O
import whole_array as WA

GRAPHS = [
    ("two_cliques5", gg.two_cliques(5)),
    ("ring30x5", gg.ring_of_cliques(30, 5)),
    ("star300", gg.star(300)),
    ("isolated", gg.isolated_and_loops(50)),
    ("single", gg.from_edges(1, [], [])),
    ("sbm8x100", gg.sbm_planted(n_blocks=8, block_size=100, p_in=0.1, p_out=0.005, seed=4)),
    ("rmat10", gg.rmat(scale=10, seed=5)),
    ("ties", gg.random_small(300, 0.03, 11, wmax=1)),
    ("rand", gg.random_small(120, 0.12, 101, wmax=6, loops=0.2)),
]
IDS = [n for n, _ in GRAPHS]


def _states(g, seed):
    rng = np.random.default_rng(seed)
    yield O.rootlabel(O.assign(g))
    a = rng.integers(0, max(g.n, 1), size=g.n).astype(np.int32)
    yield O.rootlabel(a)
    a, root, _ = O.positive(g, O.assign(g))
    yield root


@pytest.mark.parametrize("name,g", GRAPHS, ids=IDS)
def test_assign_equals_oracle(name, g):
    a, s, m = WA.expected_assign(g)
    so, mo = O.strengths(g)
    assert m == mo and np.array_equal(s, so)
    assert np.array_equal(a, O.assign(g).astype(np.int64))


@pytest.mark.parametrize("name,g", GRAPHS, ids=IDS)
def test_scan_equals_oracle(name, g):
    s, m = O.strengths(g)
    for root in _states(g, 7):
        best, gain, gl = WA.expected_scan(g, root, s.astype(np.int64), m)
        ob, og, ol = O.scan(g, root)
        assert np.array_equal(best, ob.astype(np.int64)), name
        assert np.array_equal(gain, og) and np.array_equal(gl, ol), name


def test_planted_mistakes_are_caught():
    # singletons on a path with unit weights: every interior node sees two
    # neighbouring communities with equal scores, so the tie rule decides
    g = gg.path(300)
    s, m = O.strengths(g)
    root = np.arange(g.n, dtype=np.int32)
    ob, og, ol = O.scan(g, root)
    saved = WA.best_per_group

    def largest_name(grp, score, name):   # ties to the largest name
        r, t, p = saved(grp, score, -name)
        return r, t, -p

    WA.best_per_group = largest_name
    try:
        b2, _, _ = WA.expected_scan(g, root, s.astype(np.int64), m)
    finally:
        WA.best_per_group = saved
    assert not np.array_equal(b2, ob.astype(np.int64))
    b1, _, _ = WA.expected_scan(g, root, s.astype(np.int64), m)
    assert np.array_equal(b1, ob.astype(np.int64))
    # a self-loop counted as weight to the node's own community would change g
    gl_loops = gg.random_small(120, 0.12, 101, wmax=6, loops=0.5)
    s3, m3 = O.strengths(gl_loops)
    r3 = O.rootlabel(O.assign(gl_loops))
    _, _, l3 = O.scan(gl_loops, r3)
    i = WA._rows(gl_loops)
    on_diag = gl_loops.col == i
    loop_w = np.bincount(i[on_diag], weights=gl_loops.w[on_diag], minlength=gl_loops.n).astype(np.int64)
    _, _, e3 = WA.expected_scan(gl_loops, r3, s3.astype(np.int64), m3)
    assert np.array_equal(e3, l3)
    assert loop_w.any() and not np.array_equal(e3 + m3 * loop_w, l3)
