"""CPU oracle of the Synchronised Louvain Method (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library's product path never does.

The arithmetic lives in ``slm_oracle.c`` (plain single-threaded C, each
function citing the paper's passage); this module compiles it with gcc on
first use and exposes it through ctypes with numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "slm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liborc.so")
_lock = threading.Lock()
_lib = None

FLAG_NO_POSITIVE = 1
P_ALWAYS = 1 << 32
P_HALF = 1 << 31


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain gcc, no GPU code)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
            i32, i64, u64, vp = C.c_int32, C.c_int64, C.c_uint64, C.c_void_p
            sig = {
                "orc_mix64": (u64, [u64]),
                "orc_draw": (C.c_uint32, [u64, i32, i32, i32]),
                "orc_strengths": (i64, [i32, i32p, i32p, i32p, i64p]),
                "orc_modularity_num": (i64, [i32, i32p, i32p, i32p, i32p]),
                "orc_modularity": (C.c_double, [i32, i32p, i32p, i32p, i32p]),
                "orc_assign": (None, [i32, i32p, i32p, i32p, i64p, i64, i32p]),
                "orc_rootlabel": (None, [i32, i32p, i32p]),
                "orc_sigma": (None, [i32, i32p, i64p, i64p]),
                "orc_scan": (None, [i32, i32p, i32p, i32p, i64p, i64, i32p, i64p, i32p, i64p, i64p]),
                "orc_branch_gain": (i64, [i32, i32p, i32p, i32p, i64p, i64, i32p, i32p, i64p, i32, i32]),
                "orc_target": (i32, [i32p, i32p, i32p, i64p, i64, i32p, i32, i32]),
                "orc_positive": (i32, [i32, i32p, i32p, i32p, i64p, i64, i32p, i32p]),
                "orc_compact": (i32, [i32, i32p, i32p]),
                "orc_aggregate": (i32, [i32, i32p, i32p, i32p, i32p, i32, i32p, i32p, i32p]),
                "orc_slm": (vp, [i32, i32p, i32p, i32p, u64, u64, i32, i32, C.c_uint32]),
                "orc_run_levels": (i32, [vp]),
                "orc_run_level_n": (i32, [vp, i32]),
                "orc_run_level_K": (i32, [vp, i32]),
                "orc_run_level_labels": (None, [vp, i32, i32p]),
                "orc_run_final_labels": (None, [vp, i32p]),
                "orc_run_level_stats": (None, [vp, i32, i64p]),
                "orc_run_trace_len": (i64, [vp]),
                "orc_run_trace": (None, [vp, i64p]),
                "orc_run_top": (None, [vp, i32p]),
                "orc_run_free": (None, [vp]),
                "ord_strengths": (i64, [i32, i32p, i32p, i32p, i64p, i64p]),
                "ord_symmetrise": (i32, [i32, i32p, i32p, i32p, i32p, i32p, i32p]),
                "ord_modularity_num": (i64, [i32, i32p, i32p, i32p, i32p]),
                "ord_modularity": (C.c_double, [i32, i32p, i32p, i32p, i32p]),
                "ord_assign": (None, [i32, i32p, i32p, i32p, i64p, i64p, i64, i32p]),
                "ord_sigma": (None, [i32, i32p, i64p, i64p, i64p, i64p]),
                "ord_scan": (None, [i32, i32p, i32p, i32p, i64p, i64p, i64, i32p, i64p, i64p,
                                    i32p, i64p, i64p]),
                "ord_branch_gain": (i64, [i32, i32p, i32p, i32p, i64p, i64p, i64, i32p, i32p,
                                          i64p, i64p, i32, i32]),
                "ord_target": (i32, [i32p, i32p, i32p, i64p, i64p, i64, i32p, i32, i32]),
                "ord_positive": (i32, [i32, i32p, i32p, i32p, i64p, i64p, i64, i32p, i32p]),
                "ord_slm": (vp, [i32, i32p, i32p, i32p, u64, u64, i32, i32, C.c_uint32]),
                "orc_louvain": (vp, [i32, i32p, i32p, i32p, i32, i32]),
                "orc_colour": (i32, [i32, i32p, i32p, u64, i32, i32p]),
                "orc_louvain_colour": (vp, [i32, i32p, i32p, i32p, u64, i32, i32]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    w = np.ascontiguousarray(g.w, dtype=np.int32)
    return int(g.n), rp, col, w


def _i32(x):
    return np.ascontiguousarray(x, dtype=np.int32)


def _i64(x):
    return np.ascontiguousarray(x, dtype=np.int64)


def mix64(z: int) -> int:
    return int(_load().orc_mix64(z))


def draw(seed: int, level: int, sweep: int, i: int) -> int:
    return int(_load().orc_draw(seed, level, sweep, i))


def strengths(g):
    n, rp, col, w = _csr(g)
    s = np.zeros(max(n, 1), np.int64)
    m = _load().orc_strengths(n, rp, col, w, s)
    return s[:n], int(m)


def modularity_num(g, labels) -> int:
    n, rp, col, w = _csr(g)
    return int(_load().orc_modularity_num(n, rp, col, w, _i32(labels)))


def modularity(g, labels) -> float:
    n, rp, col, w = _csr(g)
    return float(_load().orc_modularity(n, rp, col, w, _i32(labels)))


def assign(g):
    n, rp, col, w = _csr(g)
    s, m = strengths(g)
    a = np.zeros(max(n, 1), np.int32)
    _load().orc_assign(n, rp, col, w, _i64(s if n else np.zeros(1)), m, a)
    return a[:n]


def rootlabel(a):
    a = _i32(a)
    n = a.shape[0]
    root = np.zeros(max(n, 1), np.int32)
    _load().orc_rootlabel(n, a if n else np.zeros(1, np.int32), root)
    return root[:n]


def sigma(root, s):
    root = _i32(root)
    n = root.shape[0]
    out = np.zeros(max(n, 1), np.int64)
    _load().orc_sigma(n, root, _i64(s), out)
    return out[:n]


def scan(g, root, sig=None):
    """(best, gain, g) of every node for the communities named by ``root``."""
    n, rp, col, w = _csr(g)
    s, m = strengths(g)
    root = _i32(root)
    if sig is None:
        sig = sigma(root, s)
    best = np.zeros(n, np.int32)
    gain = np.zeros(n, np.int64)
    gl = np.zeros(n, np.int64)
    _load().orc_scan(n, rp, col, w, _i64(s), m, root, _i64(sig), best, gain, gl)
    return best, gain, gl


def branch_gain(g, a, root, i: int, B: int, sig=None) -> int:
    n, rp, col, w = _csr(g)
    s, m = strengths(g)
    root = _i32(root)
    if sig is None:
        sig = sigma(root, s)
    return int(_load().orc_branch_gain(n, rp, col, w, _i64(s), m, _i32(a), root, _i64(sig), i, B))


def target(g, root, i: int, B: int) -> int:
    n, rp, col, w = _csr(g)
    s, m = strengths(g)
    return int(_load().orc_target(rp, col, w, _i64(s), m, _i32(root), i, B))


def positive(g, a, root=None):
    """Run POSITIVE; returns (a, root, number of splits)."""
    n, rp, col, w = _csr(g)
    s, m = strengths(g)
    a = _i32(a).copy()
    root = rootlabel(a) if root is None else _i32(root).copy()
    k = _load().orc_positive(n, rp, col, w, _i64(s), m, a, root)
    return a, root, int(k)


def compact(root):
    root = _i32(root)
    n = root.shape[0]
    idv = np.zeros(max(n, 1), np.int32)
    K = _load().orc_compact(n, root, idv)
    return idv[:n], int(K)


def aggregate(g, idv, K: int):
    """AGGREGATE of the graph by ids in [0, K); returns a graphgen.CSR."""
    from graphgen import CSR
    n, rp, col, w = _csr(g)
    rp2 = np.zeros(K + 1, np.int32)
    col2 = np.zeros(max(g.nnz, 1), np.int32)
    w2 = np.zeros(max(g.nnz, 1), np.int32)
    nnz = _load().orc_aggregate(n, rp, col, w, _i32(idv), K, rp2, col2, w2)
    return CSR(K, rp2, col2[:nnz].copy(), w2[:nnz].copy())


class Run:
    """Result of a full oracle run (Algorithm 1)."""

    def __init__(self, levels, final, stats, trace, top):
        self.levels = levels          # list of (labels int32[n_t], K_t)
        self.final = final            # composed labels on the input nodes
        self.stats = stats            # per level: sweeps, status, moves, splits, cands, edges
        self.trace = trace            # per sweep: level, sweep, cand, pos, acc, splits
        self.top = top                # (status, sweeps) of the last unrecorded level, level-limit flag

    @property
    def num_levels(self) -> int:
        return len(self.levels)


def slm(g, seed: int = 1, P: int = P_HALF, max_sweeps: int = 1000, max_levels: int = 64,
        flags: int = 0) -> Run:
    n, rp, col, w = _csr(g)
    lib = _load()
    return _collect(lib, lib.orc_slm(n, rp, col, w, seed, P, max_sweeps, max_levels, flags), n)


def louvain(g, max_passes: int = 1000, max_levels: int = 64) -> Run:
    """Classical sequential-move Louvain on a symmetric graph, for comparison
    (stats per level: passes, 0, moves, 0, 0, entries scanned)."""
    n, rp, col, w = _csr(g)
    lib = _load()
    return _collect(lib, lib.orc_louvain(n, rp, col, w, max_passes, max_levels), n)


def colouring(g, seed: int = 1, level: int = 0):
    """First-fit colouring of g's nodes in the key order of level `level`
    (colour-synchronous Louvain); returns (colours, number of colours)."""
    n, rp, col, w = _csr(g)
    c = np.zeros(max(n, 1), np.int32)
    k = _load().orc_colour(n, rp, col, seed, level, c)
    return c[:n], int(k)


def louvain_colour(g, seed: int = 1, max_passes: int = 1000, max_levels: int = 64) -> Run:
    """Colour-synchronous Louvain on a symmetric graph: per pass the colour
    classes in turn, every node of a class moving at once; a level ends at a
    pass without moves (status 0), with a numerator gain of at most
    floor(m_w^2 / 2^20) (status 1) or at the pass limit (status 2).  Stats
    per level: passes, status, moves, 0, 0, entries scanned."""
    n, rp, col, w = _csr(g)
    lib = _load()
    return _collect(lib, lib.orc_louvain_colour(n, rp, col, w, seed, max_passes, max_levels), n)


def _collect(lib, h, n) -> Run:
    try:
        L = lib.orc_run_levels(h)
        levels = []
        stats = []
        for l in range(L):
            nl = lib.orc_run_level_n(h, l)
            lab = np.zeros(max(nl, 1), np.int32)
            lib.orc_run_level_labels(h, l, lab)
            levels.append((lab[:nl], int(lib.orc_run_level_K(h, l))))
            st = np.zeros(6, np.int64)
            lib.orc_run_level_stats(h, l, st)
            stats.append(tuple(int(x) for x in st))
        final = np.zeros(max(n, 1), np.int32)
        lib.orc_run_final_labels(h, final)
        nt = lib.orc_run_trace_len(h)
        tr = np.zeros(max(nt, 1) * 6, np.int64)
        lib.orc_run_trace(h, tr)
        top = np.zeros(3, np.int32)
        lib.orc_run_top(h, top)
        return Run(levels, final[:n], stats, tr[: nt * 6].reshape(nt, 6), tuple(int(x) for x in top))
    finally:
        lib.orc_run_free(h)


# ---------------------------------------------------------------------------
# Directed graphs (the ord_* functions): g is any CSR with sorted unique
# columns and positive weights, W_ij stored in row i.  Values are the exact
# change of the directed modularity numerator; m_w must stay below 2^30.
# ---------------------------------------------------------------------------
def directed_strengths(g):
    """(s_out, s_in, m_w) of a directed CSR."""
    n, rp, col, w = _csr(g)
    so = np.zeros(max(n, 1), np.int64)
    si = np.zeros(max(n, 1), np.int64)
    m = _load().ord_strengths(n, rp, col, w, so, si)
    return so[:n], si[:n], int(m)


def symmetrise(g):
    """U = W + W^T as a graphgen.CSR (U_ii = 2 W_ii)."""
    from graphgen import CSR
    n, rp, col, w = _csr(g)
    rpu = np.zeros(n + 1, np.int32)
    colu = np.zeros(max(2 * g.nnz, 1), np.int32)
    wu = np.zeros(max(2 * g.nnz, 1), np.int32)
    k = _load().ord_symmetrise(n, rp, col, w, rpu, colu, wu)
    return CSR(n, rpu, colu[:k].copy(), wu[:k].copy())


def _directed(g):
    so, si, m = directed_strengths(g)
    if m >= 1 << 30:
        raise ValueError("directed oracle needs m_w < 2^30")
    u = symmetrise(g)
    n, rpu, colu, wu = _csr(u)
    pad = lambda x: _i64(x if n else np.zeros(1))  # noqa: E731
    return n, rpu, colu, wu, pad(so), pad(si), m


def directed_modularity_num(g, labels) -> int:
    n, rp, col, w = _csr(g)
    return int(_load().ord_modularity_num(n, rp, col, w, _i32(labels)))


def directed_modularity(g, labels) -> float:
    n, rp, col, w = _csr(g)
    return float(_load().ord_modularity(n, rp, col, w, _i32(labels)))


def directed_assign(g):
    n, rpu, colu, wu, so, si, m = _directed(g)
    a = np.zeros(max(n, 1), np.int32)
    _load().ord_assign(n, rpu, colu, wu, so, si, m, a)
    return a[:n]


def directed_sigma(root, so, si):
    root = _i32(root)
    n = root.shape[0]
    go = np.zeros(max(n, 1), np.int64)
    gi = np.zeros(max(n, 1), np.int64)
    _load().ord_sigma(n, root, _i64(so), _i64(si), go, gi)
    return go[:n], gi[:n]


def directed_scan(g, root):
    """(best, gain, g) of every node of a directed graph."""
    n, rpu, colu, wu, so, si, m = _directed(g)
    root = _i32(root)
    go, gi = directed_sigma(root, so[:n], si[:n])
    best = np.zeros(n, np.int32)
    gain = np.zeros(n, np.int64)
    gl = np.zeros(n, np.int64)
    _load().ord_scan(n, rpu, colu, wu, so, si, m, root, _i64(go), _i64(gi), best, gain, gl)
    return best, gain, gl


def directed_branch_gain(g, a, root, i: int, B: int) -> int:
    n, rpu, colu, wu, so, si, m = _directed(g)
    root = _i32(root)
    go, gi = directed_sigma(root, so[:n], si[:n])
    return int(_load().ord_branch_gain(n, rpu, colu, wu, so, si, m, _i32(a), root, _i64(go),
                                       _i64(gi), i, B))


def directed_target(g, root, i: int, B: int) -> int:
    n, rpu, colu, wu, so, si, m = _directed(g)
    return int(_load().ord_target(rpu, colu, wu, so, si, m, _i32(root), i, B))


def directed_positive(g, a, root=None):
    """POSITIVE on a directed graph; returns (a, root, number of splits)."""
    n, rpu, colu, wu, so, si, m = _directed(g)
    a = _i32(a).copy()
    root = rootlabel(a) if root is None else _i32(root).copy()
    k = _load().ord_positive(n, rpu, colu, wu, so, si, m, a, root)
    return a, root, int(k)


def directed_slm(g, seed: int = 1, P: int = P_HALF, max_sweeps: int = 1000,
                 max_levels: int = 64, flags: int = 0) -> Run:
    """The whole method on a directed graph (entries scanned count U's entries)."""
    _directed(g)  # range check
    n, rp, col, w = _csr(g)
    lib = _load()
    return _collect(lib, lib.ord_slm(n, rp, col, w, seed, P, max_sweeps, max_levels, flags), n)
