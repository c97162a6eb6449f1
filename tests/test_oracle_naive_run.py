"""Whole runs of the C oracle against the definition-level restatement of the
method (tests/naive_slm.py) on many random tiny graphs: every level's labels,
the final partition, every level's statistics and the per-sweep trace must be
equal.  The restatement measures every decision on the modularity double sum,
so this pins the oracle's driver (sweep loop, stop reasons, synchronous write,
POSITIVE after each write, compaction, aggregation, composition) as well as
its closed-form scores."""
import numpy as np
import pytest

import graphgen as gg
import oracle as O
from brute import dense
import naive_slm

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import HealthCheck, given, settings, strategies as st  # noqa: E402


def _compare(g, seed, P, max_sweeps=30, no_positive=False, directed=False):
    levels, final, stats, trace = naive_slm.run(dense(g), O.draw, seed, P, max_sweeps=max_sweeps,
                                                no_positive=no_positive, directed=directed)
    run = O.directed_slm if directed else O.slm
    r = run(g, seed=seed, P=P, max_sweeps=max_sweeps,
            flags=O.FLAG_NO_POSITIVE if no_positive else 0)
    assert r.num_levels == len(levels)
    for (a, ka), (b, kb) in zip(r.levels, levels):
        assert ka == kb and (a == b).all()
    assert (r.final == final).all()
    assert r.stats == stats
    assert [tuple(int(x) for x in row) for row in r.trace] == trace
    return r


@st.composite
def tiny_graphs(draw):
    seed = draw(st.integers(0, 10**6))
    if draw(st.booleans()):
        # planted blocks with noise: the sweeps move many nodes and POSITIVE splits often
        blocks, size = draw(st.sampled_from([(2, 5), (2, 6), (3, 4), (3, 3), (4, 3)]))
        return gg.sbm_planted(n_blocks=blocks, block_size=size,
                              p_in=draw(st.sampled_from([0.5, 0.7, 0.9])),
                              p_out=draw(st.sampled_from([0.1, 0.2, 0.3])), seed=seed)
    n = draw(st.integers(2, 14))
    p = draw(st.sampled_from([0.2, 0.3, 0.45, 0.7]))
    wmax = draw(st.sampled_from([1, 1, 3, 6]))
    loops = draw(st.sampled_from([0.0, 0.0, 0.3]))
    return gg.random_small(n, p, seed, wmax=wmax, loops=loops)


@settings(max_examples=2000, deadline=None, suppress_health_check=[HealthCheck.too_slow])
@given(g=tiny_graphs(), seed=st.integers(0, 2**32 - 1),
       P=st.sampled_from([O.P_HALF, O.P_ALWAYS, 1 << 29, 3 << 30]))
def test_oracle_run_equals_definition_level_run(g, seed, P):
    _compare(g, seed, P)


@settings(max_examples=60, deadline=None, suppress_health_check=[HealthCheck.too_slow])
@given(g=tiny_graphs(), seed=st.integers(0, 2**32 - 1))
def test_oracle_run_without_positive_equals_definition_level_run(g, seed):
    _compare(g, seed, O.P_HALF, no_positive=True)


@st.composite
def tiny_digraphs(draw):
    return gg.random_directed(draw(st.integers(2, 12)), draw(st.sampled_from([0.2, 0.35, 0.5])),
                              draw(st.integers(0, 10**6)), wmax=draw(st.sampled_from([1, 3, 6])),
                              loops=draw(st.sampled_from([0.0, 0.3])),
                              recip=draw(st.sampled_from([0.0, 0.3, 0.8])))


@settings(max_examples=800, deadline=None, suppress_health_check=[HealthCheck.too_slow])
@given(g=tiny_digraphs(), seed=st.integers(0, 2**32 - 1),
       P=st.sampled_from([O.P_HALF, O.P_ALWAYS, 3 << 30]))
def test_directed_oracle_run_equals_definition_level_run(g, seed, P):
    _compare(g, seed, P, directed=True)


def test_the_random_cases_move_and_split():
    """The comparison is only as strong as what the runs do: over a fixed
    sample of the same graph family, sweeps move nodes, POSITIVE splits after
    moves, levels stall and aggregate."""
    rng = np.random.default_rng(1)
    moves = splits = stalled = multi = 0
    for k in range(150):
        g = (gg.sbm_planted(n_blocks=3, block_size=4, p_in=0.7, p_out=0.2, seed=k) if k % 2
             else gg.random_small(12, 0.3, 1000 + k, wmax=3))
        r = _compare(g, int(rng.integers(0, 2**32)), O.P_HALF)
        moves += sum(s[2] for s in r.stats)
        splits += sum(s[3] for s in r.stats)
        stalled += sum(s[1] == 1 for s in r.stats)
        multi += r.num_levels > 1
    assert moves > 100 and splits > 25 and stalled > 2 and multi > 15


def test_named_small_graphs_and_sweep_limit():
    moved = 0
    for g in [gg.two_cliques(4), gg.ring_of_cliques(3, 3), gg.path(8), gg.star(7),
              gg.isolated_and_loops(6), gg.random_small(10, 0.5, 3, wmax=4, loops=0.2)]:
        for P in (O.P_HALF, O.P_ALWAYS):
            r = _compare(g, 5, P)
            moved += sum(s[2] for s in r.stats)
        _compare(g, 5, O.P_HALF, max_sweeps=1)  # stops at the sweep limit
    assert moved > 0
