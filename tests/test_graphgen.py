"""The seeded input generators: the weighted LFR-style family of the paper's
experiments (Section 5.1, its table of benchmark parameters) has the degrees
and the topology and weight mixing it is asked for, and the method finds its
planted communities where they are well separated."""
import numpy as np
import pytest

import graphgen as gg
import oracle as O


def _mixing(g, comm):
    row = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    ext = comm[row] != comm[g.col]
    return ext.mean(), g.w[ext].sum() / g.w.sum()


@pytest.mark.parametrize("mu_t,mu_w", [(0.2, 0.1), (0.5, 0.4), (0.8, 0.7)])
def test_lfr_weighted_degrees_and_mixing(mu_t, mu_w):
    g, comm = gg.lfr_weighted(40000, mu_t, mu_w)
    deg = np.diff(g.row_ptr)
    assert deg.max() <= 100                  # duplicates only merge entries
    assert abs(deg.mean() - 50) < 3
    # symmetric, positive integer weights
    row = np.repeat(np.arange(g.n), deg)
    fwd = dict(zip(zip(row.tolist(), g.col.tolist()), g.w.tolist()))
    assert all(fwd[(j, i)] == w for (i, j), w in list(fwd.items())[:20000])
    assert g.w.min() >= 1
    # community sizes in [100, 1000] (the last one may absorb a remainder)
    sizes = np.bincount(comm)
    assert sizes.min() >= 100 and np.sort(sizes)[-2] <= 1000
    # external edges: mu_t less the stubs that pair inside their own
    # community by chance; external weight share close to mu_w
    e_frac, w_frac = _mixing(g, comm)
    assert mu_t - 0.05 < e_frac <= mu_t + 0.01
    assert abs(w_frac - mu_w) < 0.05


def test_lfr_weighted_is_seeded():
    a, ca = gg.lfr_weighted(5000, 0.5, 0.4, seed=9)
    b, cb = gg.lfr_weighted(5000, 0.5, 0.4, seed=9)
    assert np.array_equal(a.col, b.col) and np.array_equal(a.w, b.w) and np.array_equal(ca, cb)


@pytest.mark.parametrize("mu_t,mu_w", [(0.2, 0.1), (0.5, 0.4)])
def test_oracle_recovers_planted_lfr_communities(mu_t, mu_w):
    g, comm = gg.lfr_weighted(10000, mu_t, mu_w)
    r = O.slm(g, seed=1, P=O.P_HALF)
    lab = r.final
    # the same partition up to names: every planted community is one label
    pairs = np.unique(np.stack([comm, lab]), axis=1)
    assert pairs.shape[1] == np.unique(comm).shape[0] == np.unique(lab).shape[0]


def test_lfr_directed_orientation_and_mixing():
    g, comm = gg.lfr_directed(20000, 0.5, 0.4, recip=0.3)
    W_rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    pairs = set(zip(W_rows.tolist(), g.col.tolist()))
    both = sum((j, i) in pairs for (i, j) in pairs) / len(pairs)
    assert 0.3 < both < 0.6  # some arcs come with their reverse, most do not
    ext = comm[W_rows] != comm[g.col]
    assert abs(g.w[ext].sum() / g.w.sum() - 0.4) < 0.06
    so, si, m = O.directed_strengths(g)
    assert so.sum() == si.sum() == m and not (so == si).all()
    a, ca = gg.lfr_directed(3000, 0.2, 0.1, seed=4)
    b, cb = gg.lfr_directed(3000, 0.2, 0.1, seed=4)
    assert np.array_equal(a.col, b.col) and np.array_equal(a.w, b.w) and np.array_equal(ca, cb)
