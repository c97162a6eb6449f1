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
    h = lib.orc_slm(n, rp, col, w, seed, P, max_sweeps, max_levels, flags)
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
