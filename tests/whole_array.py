"""Whole-array recomputations of ASSIGN and of the MAXIMAL scan for graphs
of millions of nodes (vectorised numpy, exact int64), used by the full-size
GPU tests to compare every node's output instead of a sample.

Each function restates its step's definition directly: group the entries by
node, take the largest score per node, ties to the smallest name.  They share nothing with the oracle or
with the CUDA library; tests/test_whole_array.py pins them against brute force
and the oracle on small graphs.
"""
import numpy as np


def _rows(g):
    return np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))


def strengths(g):
    return np.bincount(_rows(g), weights=g.w, minlength=g.n).astype(np.int64)  # exact: m_w < 2^31


def best_per_group(grp, score, name):
    """For entries grouped by grp (sorted, non-decreasing) with names unique
    within a group: (group, best score, name) of every group, the best being
    the largest score with ties to the smallest name."""
    starts = np.flatnonzero(np.r_[True, grp[1:] != grp[:-1]])
    sizes = np.diff(np.r_[starts, grp.shape[0]])
    top = np.maximum.reduceat(score, starts)
    at_top = score == np.repeat(top, sizes)
    big = np.iinfo(np.int64).max
    pick = np.minimum.reduceat(np.where(at_top, name, big), starts)
    return grp[starts], top, pick


def expected_assign(g):
    """ASSIGN (Section 3.1) of every node: argmax_j (m_w W_ij - s_i s_j) over
    neighbours j != i, ties to the smallest j, itself when the best is <= 0."""
    s = strengths(g)
    m = int(s.sum())
    i = _rows(g)
    j = g.col.astype(np.int64)
    wv = g.w.astype(np.int64)
    keep = j != i
    i, j, wv = i[keep], j[keep], wv[keep]
    sc = m * wv - s[i] * s[j]
    a = np.arange(g.n, dtype=np.int64)
    if i.shape[0]:
        rows, top, pick = best_per_group(i, sc, j)     # CSR order: grouped by row
        good = top > 0
        a[rows[good]] = pick[good]
    return a, s, m


def expected_scan(g, root, s, m):
    """MAXIMAL's per-node half (Section 3.4) for every node: the weight to each
    neighbouring community, the best other community by m_w k_{i,C} - s_i
    Sigma_C (ties smallest C), its gain over staying, and the local gain g."""
    root = root.astype(np.int64)
    sigma = np.bincount(root, weights=s, minlength=g.n).astype(np.int64)
    i = _rows(g)
    j = g.col.astype(np.int64)
    keep = j != i
    i, c, wv = i[keep], root[j[keep]], g.w[keep].astype(np.int64)
    key = i * np.int64(g.n) + c
    uk, inv = np.unique(key, return_inverse=True)
    k = np.bincount(inv, weights=wv).astype(np.int64)
    ui, uc = uk // g.n, uk % g.n
    ci = root
    own = np.zeros(g.n, np.int64)
    is_own = uc == ci[ui]
    own[ui[is_own]] = k[is_own]
    g_loc = m * own - s * (sigma[ci] - s)
    best = ci.copy()
    gain = np.zeros(g.n, np.int64)
    oth = ~is_own
    oi, oc, ok = ui[oth], uc[oth], k[oth]
    if oi.shape[0]:
        sc = m * ok - s[oi] * sigma[oc]
        rows, top, pick = best_per_group(oi, sc, oc)   # np.unique sorted by (i, C)
        gn = top - g_loc[rows]
        pos = gn > 0
        best[rows[pos]] = pick[pos]
        gain[rows[pos]] = gn[pos]
    return best, gain, g_loc
