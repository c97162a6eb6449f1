"""Definition-level helpers for the oracle's pins (dense, tiny graphs only).

Nothing here reuses the oracle's formulas: modularity is the double sum of the
weighted modularity definition (Section 2.4) over all node pairs, and every
gain is measured as a difference of that sum before and after a change.
"""
import numpy as np


def dense(g):
    W = np.zeros((g.n, g.n), dtype=np.int64)
    for u in range(g.n):
        for p in range(g.row_ptr[u], g.row_ptr[u + 1]):
            W[u, g.col[p]] += g.w[p]
    return W


def q_num_def(W, labels):
    """sum_{i,j} (m_w W_ij - s_i s_j) delta(c_i, c_j): m_w^2 times Q_w."""
    labels = np.asarray(labels)
    s = W.sum(axis=1)
    m = int(W.sum())
    same = labels[:, None] == labels[None, :]
    return int((m * W - np.outer(s, s))[same].sum())


def set_partitions(n):
    """All set partitions of {0..n-1} as restricted growth strings, shape [Bell(n), n]."""
    if n == 0:
        return np.zeros((1, 0), dtype=np.int8)
    parts = np.zeros((1, 1), dtype=np.int8)
    for k in range(1, n):
        mx = parts.max(axis=1)
        rows = []
        for v in range(0, k + 1):
            ok = mx + 1 >= v
            sel = parts[ok]
            rows.append(np.concatenate([sel, np.full((sel.shape[0], 1), v, np.int8)], axis=1))
        parts = np.concatenate(rows, axis=0)
    return parts


def brute_max_q_num(W):
    """Largest m_w^2 Q over every partition (exhaustive, n <= 10)."""
    n = W.shape[0]
    P = set_partitions(n)
    s = W.sum(axis=1)
    m = int(W.sum())
    C = m * W - np.outer(s, s)
    tot = np.zeros(P.shape[0], dtype=np.int64)
    for i in range(n):
        for j in range(n):
            if C[i, j]:
                tot += C[i, j] * (P[:, i] == P[:, j])
    k = int(np.argmax(tot))
    return int(tot[k]), P[k]


def tail(a, i):
    """Nodes whose forward path in the assignment graph reaches i (brute force)."""
    n = len(a)
    out = []
    for v in range(n):
        x = v
        for _ in range(n + 1):
            if x == i:
                out.append(v)
                break
            x = a[x]
    return out


def components(a):
    """Community names by brute force: follow n steps to land on the cycle, then
    name the component by the cycle's minimum node."""
    n = len(a)
    root = np.zeros(n, dtype=np.int64)
    for v in range(n):
        x = v
        for _ in range(n):
            x = a[x]
        cyc = [x]
        y = a[x]
        while y != x:
            cyc.append(y)
            y = a[y]
        root[v] = min(cyc)
    return root


def q_num_def_directed(W, labels):
    """sum_{i,j} (m_w W_ij - s_i^out s_j^in) delta(c_i, c_j) for any (directed)
    W: m_w^2 times the directed Q_w of Section 2.4."""
    labels = np.asarray(labels)
    so = W.sum(axis=1)
    si = W.sum(axis=0)
    m = int(W.sum())
    same = labels[:, None] == labels[None, :]
    return int((m * W - np.outer(so, si))[same].sum())


def brute_max_q_num_directed(W):
    """Largest m_w^2 Q of a directed W over every partition (exhaustive, n <= 9)."""
    n = W.shape[0]
    P = set_partitions(n)
    m = int(W.sum())
    C = m * W - np.outer(W.sum(axis=1), W.sum(axis=0))
    tot = np.zeros(P.shape[0], dtype=np.int64)
    for i in range(n):
        for j in range(n):
            if C[i, j]:
                tot += C[i, j] * (P[:, i] == P[:, j])
    k = int(np.argmax(tot))
    return int(tot[k]), P[k]
