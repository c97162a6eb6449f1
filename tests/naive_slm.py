"""The whole Synchronised Louvain Method restated at definition level for tiny
graphs (a naive second oracle, test infrastructure only).

Every decision is measured on the modularity numerator's double sum
(brute.q_num_def): a node's best community, its gain and local gain, a
branch's gain, a move's target and every POSITIVE split are differences of
that sum before and after the change, never the closed-form scores of the C
oracle.  The acceptance draw is an input (the oracle's splitmix64 draw, pinned
on its own against the published outputs).  The sweep loop, stop reasons,
synchronous write, POSITIVE after each write, compaction, AGGREGATE and
composition follow Algorithm 1 and the readings the C oracle takes.  With
directed=True the same run uses the directed numerator (Section 2.4's Q_w with
out- and in-strengths), the reference of the oracle's ord_slm.
"""
import numpy as np

from brute import components, q_num_def, q_num_def_directed, tail

# the numerator in use: the symmetric one, or the directed one (run(directed=True))
_NUM = [q_num_def]


def _move_gain(W, root, idx, C):
    lab = root.copy()
    lab[idx] = C
    return _NUM[0](W, lab) - _NUM[0](W, root)


def _pair_gain(W, i, j):
    """Gain of i joining {j} from the all-singleton state."""
    single = np.arange(W.shape[0])
    lab = single.copy()
    lab[i] = j
    return _NUM[0](W, lab) - _NUM[0](W, single)


def _nbrs(W, i):
    """Neighbours of i: nodes joined to it by an entry in either direction."""
    return [int(j) for j in np.flatnonzero(W[i] + W[:, i]) if j != i]


def assign(W):
    n = W.shape[0]
    a = np.arange(n)
    for i in range(n):
        nb = _nbrs(W, i)
        if not nb:
            continue
        g = {j: _pair_gain(W, i, j) for j in nb}
        top = max(g.values())
        if top > 0:
            a[i] = min(j for j in nb if g[j] == top)
    return a


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


def positive(W, a):
    """POSITIVE; returns (a, number of splits)."""
    n = W.shape[0]
    a = a.copy()
    splits = 0
    while True:
        root = components(a)
        flagged = None
        for A in sorted(set(root.tolist())):
            for i in np.flatnonzero(root == A):
                if _move_gain(W, root, [i], n + 1) > 0:  # leaving raises Q: g(i) < 0
                    flagged = A
                    break
            if flagged is not None:
                break
        if flagged is None:
            return a, splits
        q0 = _NUM[0](W, root)
        best = None
        for ty, u, v, b in _split_options(a, root, flagged):
            d = _NUM[0](W, components(b)) - q0
            key = (-d, ty, u, v)
            if best is None or key < best[0]:
                best = (key, b)
        a = best[1]
        splits += 1


def run(W0, draw, seed, P, max_sweeps=1000, max_levels=64, no_positive=False, directed=False):
    """Levels [(ids, K)], final labels, per-level stats (sweeps, status, moves,
    splits, candidates, entries scanned) and the per-sweep trace.  With
    directed=True, W0 is any (directed) weight matrix: the directed numerator
    decides, neighbours are joined in either direction, and the entries
    scanned per sweep are those of W + W^T."""
    _NUM[0] = q_num_def_directed if directed else q_num_def
    try:
        return _run(W0, draw, seed, P, max_sweeps, max_levels, no_positive)
    finally:
        _NUM[0] = q_num_def


def _run(W0, draw, seed, P, max_sweeps, max_levels, no_positive):
    n0 = W0.shape[0]
    final = np.arange(n0)
    levels, stats, trace = [], [], []
    W = W0.copy()
    t = 0
    while True:
        n = W.shape[0]
        nnz = int(np.count_nonzero(W + W.T))  # = entries of W when W is symmetric
        a = assign(W)
        splits = moves = cands = edges = 0
        if not no_positive:
            a, k = positive(W, a)
            splits += k
        status, sweep = 2, 0
        while sweep < max_sweeps:
            root = components(a)
            edges += nnz
            best = np.array(root)
            gain = np.zeros(n, np.int64)
            for i in range(n):
                d = {}
                for j in _nbrs(W, i):
                    C = int(root[j])
                    if C != root[i] and C not in d:
                        d[C] = _move_gain(W, root, [i], C)
                if d and max(d.values()) > 0:
                    top = max(d.values())
                    best[i] = min(C for C in d if d[C] == top)
                    gain[i] = top
            cand = [i for i in range(n) if gain[i] > 0]
            cands += len(cand)
            if not cand:
                status = 0
                trace.append((t, sweep, 0, 0, 0, 0))
                sweep += 1
                break
            pos = [i for i in cand if _move_gain(W, root, tail(a, i), int(best[i])) > 0]
            if not pos:
                status = 1
                trace.append((t, sweep, len(cand), 0, 0, 0))
                sweep += 1
                break
            acc = [i for i in pos if draw(seed, t, sweep, i) < P]
            tgt = {}
            for i in acc:
                js = [j for j in _nbrs(W, i) if root[j] == best[i]]
                g = {j: _pair_gain(W, i, j) for j in js}
                top = max(g.values())
                tgt[i] = min(j for j in js if g[j] == top)
            for i in acc:
                a[i] = tgt[i]
            moves += len(acc)
            spl = 0
            if acc and not no_positive:
                a, spl = positive(W, a)
                splits += spl
            trace.append((t, sweep, len(cand), len(pos), len(acc), spl))
            sweep += 1
        root = components(a)
        names = np.unique(root)
        K = names.shape[0]
        ids = np.searchsorted(names, root)
        if K == n:
            return levels, final, stats, trace
        levels.append((ids, K))
        stats.append((sweep, status, moves, splits, cands, edges))
        final = ids[final]
        Pm = np.zeros((n, K), np.int64)
        Pm[np.arange(n), ids] = 1
        W = Pm.T @ W @ Pm
        t += 1
        if t >= max_levels:
            return levels, final, stats, trace
