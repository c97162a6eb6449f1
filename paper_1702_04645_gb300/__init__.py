"""GB300 (sm_103a) implementation of the Synchronised Louvain Method.

Python binding of the C ABI in ``include/slm.h`` and ``include/slm_steps.h``:
argument marshalling only.  Every step of the method runs in the CUDA kernels
of ``libslm.so``; there is no CPU fallback, and importing any entry point
raises when the library has not been built (see ``build()``).

PyTorch provides device memory and streams for the step functions; the
graph-level API accepts numpy arrays (host memory) or CUDA tensors.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from .build_lib import LIB, build  # noqa: F401

__all__ = ["Graph", "Batch", "Server", "pack_forest", "get_scan_tuning", "set_scan_tuning", "Options", "LevelStats", "SlmError", "build", "load", "step_strengths",
           "step_assign", "step_components", "step_scan", "step_branch_gain", "step_maximal",
           "step_positive", "step_compact", "step_aggregate", "step_modularity",
           "FLAG_NO_POSITIVE", "FLAG_STRICT", "P_HALF", "P_ALWAYS"]

SLM_HOST = 0
SLM_DEVICE = 1
FLAG_NO_POSITIVE = 1
FLAG_STRICT = 2
FLAG_TIMING = 4
PHASES = ["assign", "components", "positive", "scan", "move", "level", "sigma",
          "positive_rounds"]
SCAN_BUCKETS = ["isolated", "deg1_4", "deg5_8", "deg9_16", "deg17_32", "deg33_256",
                "deg257_1024", "deg1025_2048", "deg2049_4096", "hubs"]
POSITIVE_PHASES = ["setup", "offsets", "walks_edges", "credits", "best_cut", "apply_cut",
                   "components", "local_gains", "next_list", "full_grid_rounds",
                   "full_grid_visits"]
P_HALF = 1 << 31
P_ALWAYS = 1 << 32

STATUS = {0: "SLM_OK", 1: "SLM_ERR_INVALID_ARGUMENT", 2: "SLM_ERR_NOT_SYMMETRIC",
          3: "SLM_ERR_OVERFLOW", 4: "SLM_ERR_OUT_OF_MEMORY", 5: "SLM_ERR_CUDA",
          6: "SLM_ERR_NOT_RUN", 7: "SLM_ERR_NOT_CONVERGED", 8: "SLM_ERR_TIMEOUT",
          9: "SLM_ERR_BUDGET", 10: "SLM_ERR_CANCELLED", 11: "SLM_ERR_DEADLINE"}

# every exported entry point, as declared in include/*.h
EXPORTS = ["slm_default_options", "slm_create_graph", "slm_create_graph_directed",
           "slm_graph_is_directed", "slm_run", "slm_run_louvain", "slm_num_levels",
           "slm_get_partition", "slm_modularity", "slm_get_stats", "slm_modularity_of",
           "slm_destroy_graph", "slm_status_string", "slm_last_error", "slm_step_strengths",
           "slm_step_assign", "slm_step_components", "slm_step_scan", "slm_step_branch_gain",
           "slm_step_maximal", "slm_step_positive", "slm_step_compact", "slm_step_aggregate",
           "slm_step_modularity", "slm_get_trace", "slm_get_timing", "slm_get_positive_profile", "slm_get_scan_timing", "slm_get_scan_bucket_timing", "slm_set_scan_tuning",
           "slm_get_scan_tuning", "slm_release_cached_memory", "slm_check_grid_barrier",
           "slm_launch_count", "slm_debug_fail_allocation",
           "slm_step_modularity_noalloc", "slm_batch_create", "slm_batch_run",
           "slm_batch_num_graphs", "slm_batch_num_levels", "slm_batch_get_partition",
           "slm_batch_modularity", "slm_batch_get_stats", "slm_batch_run_info",
           "slm_batch_destroy", "slm_batch_last_error", "slm_server_footprint", "slm_server_create",
           "slm_server_submit", "slm_server_submit_deadline", "slm_server_submit_directed", "slm_server_cancel", "slm_server_poll", "slm_server_wait", "slm_server_request_info",
           "slm_server_result", "slm_server_get_stats", "slm_server_destroy",
           "slm_server_last_error"]


def launch_count() -> int:
    """Kernels launched by the library in this process so far."""
    return int(load().slm_launch_count())


class SlmError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{self.name}: {msg}" if msg else self.name)


class GraphDesc(C.Structure):
    _fields_ = [("n", C.c_int32), ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p),
                ("weights", C.c_void_p)]


class RequestInfo(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("n", C.c_int32),
                ("n_communities", C.c_int32), ("nnz", C.c_int64), ("levels", C.c_int32),
                ("slot", C.c_int32), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double), ("modularity", C.c_double), ("footprint", C.c_uint64),
                ("peak_bytes", C.c_uint64), ("edges_scanned", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("rejected", C.c_int64), ("queued", C.c_int32), ("running", C.c_int32),
                ("max_running", C.c_int32), ("budget_bytes", C.c_uint64),
                ("reserved_bytes", C.c_uint64), ("max_reserved_bytes", C.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3


class ScanTuning(C.Structure):
    _fields_ = [("streams", C.c_int32), ("blocks_large", C.c_int32), ("blocks_mid", C.c_int32),
                ("blocks_small", C.c_int32), ("blocks_warp", C.c_int32), ("blocks_hub", C.c_int32),
                ("blocks_group", C.c_int32), ("shape_alt", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def get_scan_tuning() -> dict:
    t = ScanTuning()
    _check(load().slm_get_scan_tuning(C.byref(t)))
    return t.as_dict()


def set_scan_tuning(**fields) -> dict:
    """Change some fields of the process-wide scan tuning; returns the new tuning."""
    cur = get_scan_tuning()
    cur.update(fields)
    t = ScanTuning(**cur)
    _check(load().slm_set_scan_tuning(C.byref(t)))
    return cur


class Options(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("accept_p32", C.c_uint64), ("max_sweeps", C.c_int32),
                ("max_levels", C.c_int32), ("flags", C.c_uint32)]


class LevelStats(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_communities", C.c_int32), ("sweeps", C.c_int32),
                ("status", C.c_int32), ("moves", C.c_int64), ("splits", C.c_int64),
                ("candidates", C.c_int64), ("edges_scanned", C.c_int64), ("nnz", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lock = threading.Lock()
_lib = None


def load():
    """Load libslm.so from the package's build folder; raise if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: build the CUDA library first "
                               "(paper_1702_04645_gb300.build())")
        lib = C.CDLL(LIB)
        vp, i32, i64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
        sig = {
            "slm_default_options": (None, [C.POINTER(Options)]),
            "slm_create_graph": (C.c_int, [i32, vp, vp, vp, C.c_int, vp, C.POINTER(vp)]),
            "slm_create_graph_directed": (C.c_int, [i32, vp, vp, vp, C.c_int, vp, C.POINTER(vp)]),
            "slm_graph_is_directed": (i32, [vp]),
            "slm_run": (C.c_int, [vp, C.POINTER(Options), vp]),
            "slm_run_louvain": (C.c_int, [vp, C.c_uint64, C.c_int32, C.c_int32, vp]),
            "slm_num_levels": (C.c_int, [vp, C.POINTER(i32)]),
            "slm_get_partition": (C.c_int, [vp, i32, vp, C.c_int, C.POINTER(i32)]),
            "slm_modularity": (C.c_int, [vp, i32, C.POINTER(C.c_double)]),
            "slm_get_stats": (C.c_int, [vp, i32, C.POINTER(LevelStats)]),
            "slm_modularity_of": (C.c_int, [vp, vp, C.c_int, C.POINTER(C.c_double)]),
            "slm_destroy_graph": (None, [vp]),
            "slm_status_string": (C.c_char_p, [C.c_int]),
            "slm_last_error": (C.c_char_p, [vp]),
            "slm_get_trace": (C.c_int, [vp, vp, i64, C.POINTER(i64)]),
            "slm_get_timing": (C.c_int, [vp, vp, vp]),
            "slm_get_positive_profile": (C.c_int, [vp, vp, i32, C.POINTER(i32)]),
            "slm_get_scan_timing": (C.c_int, [vp, i32, C.POINTER(C.c_double), C.POINTER(i64)]),
            "slm_get_scan_bucket_timing": (C.c_int, [vp, vp, i32, C.POINTER(i32)]),
            "slm_set_scan_tuning": (C.c_int, [C.POINTER(ScanTuning)]),
            "slm_get_scan_tuning": (C.c_int, [C.POINTER(ScanTuning)]),
            "slm_launch_count": (u64, []),
            "slm_debug_fail_allocation": (None, [i64]),
            "slm_release_cached_memory": (None, []),
            "slm_check_grid_barrier": (C.c_int, [i32, i32, C.c_double, vp]),
            "slm_step_strengths": (C.c_int, [i32, vp, vp, vp, vp, C.POINTER(i64), vp]),
            "slm_step_assign": (C.c_int, [i32, vp, vp, vp, vp, i64, vp, vp]),
            "slm_step_components": (C.c_int, [i32, vp, vp, vp]),
            "slm_step_scan": (C.c_int, [i32, vp, vp, vp, vp, i64, vp, vp, vp, vp, vp]),
            "slm_step_branch_gain": (C.c_int, [i32, vp, vp, vp, vp, i64, vp, vp, vp, vp, vp, vp]),
            "slm_step_maximal": (C.c_int, [i32, vp, vp, vp, vp, i64, vp, vp, u64, u64, i32, i32,
                                           vp, vp]),
            "slm_step_positive": (C.c_int, [i32, vp, vp, vp, vp, i64, vp, vp, vp, vp]),
            "slm_step_compact": (C.c_int, [i32, vp, vp, C.POINTER(i32), vp]),
            "slm_step_aggregate": (C.c_int, [i32, vp, vp, vp, vp, i32, vp, vp, vp,
                                             C.POINTER(i32), vp]),
            "slm_step_modularity": (C.c_int, [i32, vp, vp, vp, vp, C.POINTER(C.c_double),
                                              C.POINTER(i64), vp]),
            "slm_step_modularity_noalloc": (C.c_int, [i32, vp, vp, vp, vp, vp, vp, vp]),
            "slm_batch_create": (C.c_int, [i32, vp, vp, vp, vp, vp, C.c_int, vp, C.POINTER(vp)]),
            "slm_batch_run": (C.c_int, [vp, C.POINTER(Options), vp]),
            "slm_batch_num_graphs": (C.c_int, [vp, C.POINTER(i32)]),
            "slm_batch_num_levels": (C.c_int, [vp, i32, C.POINTER(i32)]),
            "slm_batch_get_partition": (C.c_int, [vp, i32, i32, vp, C.POINTER(i32)]),
            "slm_batch_modularity": (C.c_int, [vp, i32, C.POINTER(C.c_double)]),
            "slm_batch_get_stats": (C.c_int, [vp, i32, i32, C.POINTER(LevelStats)]),
            "slm_batch_run_info": (C.c_int, [vp, C.POINTER(i32), C.POINTER(i64)]),
            "slm_batch_destroy": (None, [vp]),
            "slm_batch_last_error": (C.c_char_p, [vp]),
            "slm_server_footprint": (u64, [i32, i64]),
            "slm_server_create": (C.c_int, [u64, i32, C.POINTER(vp)]),
            "slm_server_submit": (C.c_int, [vp, C.POINTER(GraphDesc), C.POINTER(Options),
                                            C.POINTER(u64)]),
            "slm_server_submit_deadline": (C.c_int, [vp, C.POINTER(GraphDesc), C.POINTER(Options),
                                                     C.c_double, C.POINTER(u64)]),
            "slm_server_submit_directed": (C.c_int, [vp, C.POINTER(GraphDesc), C.POINTER(Options),
                                                     C.c_double, C.POINTER(u64)]),
            "slm_server_cancel": (C.c_int, [vp, u64]),
            "slm_server_poll": (C.c_int, [vp, u64, C.POINTER(i32)]),
            "slm_server_wait": (C.c_int, [vp, u64, C.c_double]),
            "slm_server_request_info": (C.c_int, [vp, u64, C.POINTER(RequestInfo)]),
            "slm_server_result": (C.c_int, [vp, u64, vp, C.POINTER(i32), C.POINTER(C.c_double),
                                            i32]),
            "slm_server_get_stats": (C.c_int, [vp, C.POINTER(ServerStats)]),
            "slm_server_destroy": (None, [vp]),
            "slm_server_last_error": (C.c_char_p, [vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(st: int, handle=None):
    if st != 0:
        lib = load()
        msg = lib.slm_last_error(handle)
        raise SlmError(st, msg.decode() if msg else "")


# ---------------------------------------------------------------------------
# helpers for torch tensors (device memory and streams come from PyTorch)
# ---------------------------------------------------------------------------
def _torch():
    import torch
    return torch


def _stream(stream=None):
    if stream is not None:
        return C.c_void_p(int(stream))
    torch = _torch()
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _dev_i32(x):
    """int32 CUDA tensor of x; an empty input becomes one zero so that its
    pointer is valid (sizes are passed separately and bound every read)."""
    torch = _torch()
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x, dtype=np.int32))
    x = x.to(device="cuda", dtype=torch.int32).contiguous()
    if x.numel() == 0:
        x = torch.zeros(1, dtype=torch.int32, device="cuda")
    return x


def _empty(n, dtype):
    torch = _torch()
    return torch.empty(max(int(n), 1), dtype=dtype, device="cuda")


# ---------------------------------------------------------------------------
# Graph-level API
# ---------------------------------------------------------------------------
class Graph:
    """A graph resident on the device and the results of its last run."""

    def __init__(self, row_ptr, col, w=None, stream=None, directed: bool = False):
        """directed=True: (row_ptr, col, w) is a directed W (out-arcs per row),
        and the run optimises the directed Q_w (slm_create_graph_directed)."""
        lib = load()
        self._h = C.c_void_p()
        is_np = isinstance(row_ptr, np.ndarray)
        if is_np:
            self._keep = [np.ascontiguousarray(row_ptr, dtype=np.int32),
                          np.ascontiguousarray(col, dtype=np.int32),
                          None if w is None else np.ascontiguousarray(w, dtype=np.int32)]
            ptrs = [C.c_void_p(a.ctypes.data) if a is not None and a.size else C.c_void_p(0)
                    for a in self._keep]
            where = SLM_HOST
            st = C.c_void_p(int(stream)) if stream is not None else C.c_void_p(0)
        else:
            torch = _torch()
            self._keep = [t.contiguous() if t is not None else None for t in (row_ptr, col, w)]
            where = SLM_DEVICE if self._keep[0].is_cuda else SLM_HOST
            ptrs = [_ptr(t) if t is not None else C.c_void_p(0) for t in self._keep]
            st = _stream(stream) if where == SLM_DEVICE else C.c_void_p(0)
            del torch
        self.n = int(len(self._keep[0]) - 1)
        create = lib.slm_create_graph_directed if directed else lib.slm_create_graph
        _check(create(self.n, ptrs[0], ptrs[1], ptrs[2], where, st, C.byref(self._h)))
        self.directed = bool(directed)
        self._keep = None

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().slm_destroy_graph(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, seed: int = 1, accept_p32: int = P_HALF, max_sweeps: int = 1000,
            max_levels: int = 64, flags: int = 0, stream=None):
        o = Options(seed, accept_p32, max_sweeps, max_levels, flags)
        st = C.c_void_p(int(stream)) if stream is not None else C.c_void_p(0)
        _check(load().slm_run(self._h, C.byref(o), st), self._h)
        return self

    def run_louvain(self, seed: int = 1, max_passes: int = 1000, max_levels: int = 64,
                    stream=None):
        """Colour-synchronous Louvain (slm_run_louvain); results are read with
        the same calls as those of run()."""
        st = C.c_void_p(int(stream)) if stream is not None else C.c_void_p(0)
        _check(load().slm_run_louvain(self._h, seed, max_passes, max_levels, st), self._h)
        return self

    def num_levels(self) -> int:
        v = C.c_int32()
        _check(load().slm_num_levels(self._h, C.byref(v)), self._h)
        return v.value

    def partition(self, level: int = -1):
        """(labels as int32 numpy array, number of communities)."""
        lib = load()
        if level == -1:
            n = self.n
        else:
            n = self.stats(level).n
        out = np.zeros(max(n, 1), dtype=np.int32)
        K = C.c_int32()
        _check(lib.slm_get_partition(self._h, level, C.c_void_p(out.ctypes.data), SLM_HOST,
                                     C.byref(K)), self._h)
        return out[:n], K.value

    def partition_device(self, level: int = -1):
        """(labels as an int32 CUDA tensor, number of communities)."""
        n = self.n if level == -1 else self.stats(level).n
        out = _empty(max(n, 1), _torch().int32)
        K = C.c_int32()
        _check(load().slm_get_partition(self._h, level, _ptr(out), SLM_DEVICE, C.byref(K)),
               self._h)
        return out[:n], K.value

    def modularity(self, level: int = -1) -> float:
        q = C.c_double()
        _check(load().slm_modularity(self._h, level, C.byref(q)), self._h)
        return q.value

    def modularity_of(self, labels) -> float:
        lab = np.ascontiguousarray(labels, dtype=np.int32)
        q = C.c_double()
        _check(load().slm_modularity_of(self._h, C.c_void_p(lab.ctypes.data), SLM_HOST,
                                        C.byref(q)), self._h)
        return q.value

    def stats(self, level: int) -> LevelStats:
        s = LevelStats()
        _check(load().slm_get_stats(self._h, level, C.byref(s)), self._h)
        return s

    def timing(self):
        """{phase: (milliseconds, intervals)} of the last run made with FLAG_TIMING."""
        ms = np.zeros(8, dtype=np.float64)
        cnt = np.zeros(8, dtype=np.int64)
        _check(load().slm_get_timing(self._h, C.c_void_p(ms.ctypes.data),
                                     C.c_void_p(cnt.ctypes.data)), self._h)
        return {PHASES[k]: (float(ms[k]), int(cnt[k])) for k in range(8)}

    def scan_timing(self, level: int):
        """(milliseconds, scans) of one level's scans in the last run made with FLAG_TIMING."""
        ms = C.c_double()
        cnt = C.c_int64()
        _check(load().slm_get_scan_timing(self._h, level, C.byref(ms), C.byref(cnt)), self._h)
        return ms.value, cnt.value

    def scan_bucket_timing(self):
        """{bucket: milliseconds} of the level-0 scans of the last run made with FLAG_TIMING."""
        ms = np.zeros(len(SCAN_BUCKETS), dtype=np.float64)
        ln = C.c_int32()
        _check(load().slm_get_scan_bucket_timing(self._h, C.c_void_p(ms.ctypes.data), ms.shape[0],
                                                 C.byref(ln)), self._h)
        return {SCAN_BUCKETS[k]: float(ms[k]) for k in range(min(ln.value, ms.shape[0]))}

    def positive_profile(self):
        """{phase: milliseconds} of the POSITIVE rounds of the last run made with
        FLAG_TIMING, summed over all rounds."""
        ns = np.zeros(len(POSITIVE_PHASES), dtype=np.int64)
        ln = C.c_int32()
        _check(load().slm_get_positive_profile(self._h, C.c_void_p(ns.ctypes.data), ns.shape[0],
                                               C.byref(ln)), self._h)
        out = {POSITIVE_PHASES[k]: float(ns[k]) / 1e6 for k in range(min(ln.value, 9))}
        for k in range(9, min(ln.value, ns.shape[0])):
            out[POSITIVE_PHASES[k]] = int(ns[k])  # counts, not times
        return out

    def trace(self) -> np.ndarray:
        lib = load()
        ln = C.c_int64()
        _check(lib.slm_get_trace(self._h, C.c_void_p(0), 0, C.byref(ln)), self._h)
        out = np.zeros((max(ln.value, 1), 6), dtype=np.int64)
        _check(lib.slm_get_trace(self._h, C.c_void_p(out.ctypes.data), ln.value, C.byref(ln)),
               self._h)
        return out[: ln.value]


# ---------------------------------------------------------------------------
# Batched API: a forest of independent graphs in one run
# ---------------------------------------------------------------------------
def pack_forest(graphs):
    """Concatenate CSR graphs (objects with n, row_ptr, col, w) into one
    block-diagonal CSR; returns (graph_off, row_ptr, col, w) numpy arrays."""
    goff = np.zeros(len(graphs) + 1, dtype=np.int64)
    for k, g in enumerate(graphs):
        goff[k + 1] = goff[k] + g.n
    nnz = sum(int(g.row_ptr[-1]) for g in graphs)
    rp = np.zeros(int(goff[-1]) + 1, dtype=np.int64)
    col = np.zeros(nnz, dtype=np.int32)
    w = np.zeros(nnz, dtype=np.int32)
    e = 0
    for k, g in enumerate(graphs):
        gr = np.asarray(g.row_ptr, dtype=np.int64)
        rp[goff[k] + 1: goff[k + 1] + 1] = gr[1:] + e
        m = int(gr[-1])
        col[e:e + m] = np.asarray(g.col, dtype=np.int64) + goff[k]
        w[e:e + m] = g.w
        e += m
    if e >= 2**31 or goff[-1] >= 2**31:
        raise ValueError("forest too large for int32 CSR")
    return goff.astype(np.int32), rp.astype(np.int32), col, w


class Batch:
    """Many graphs run together (include/slm_batch.h)."""

    def __init__(self, graphs=None, *, graph_off=None, row_ptr=None, col=None, w=None,
                 seeds=None, stream=None):
        lib = load()
        if graphs is not None:
            graph_off, row_ptr, col, w = pack_forest(graphs)
        goff = np.ascontiguousarray(graph_off, dtype=np.int32)
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        cl = np.ascontiguousarray(col, dtype=np.int32)
        ww = None if w is None else np.ascontiguousarray(w, dtype=np.int32)
        sd = None if seeds is None else np.ascontiguousarray(seeds, dtype=np.uint64)
        self.G = len(goff) - 1
        self.goff = goff
        self._h = C.c_void_p()
        st = C.c_void_p(int(stream)) if stream is not None else C.c_void_p(0)
        ptr = lambda a: C.c_void_p(a.ctypes.data) if a is not None and a.size else C.c_void_p(0)  # noqa: E731
        rc = lib.slm_batch_create(self.G, ptr(goff), ptr(rp), ptr(cl), ptr(ww), ptr(sd), SLM_HOST,
                                  st, C.byref(self._h))
        if rc != 0:
            msg = lib.slm_batch_last_error(None)
            raise SlmError(rc, msg.decode() if msg else "")

    def _check(self, rc):
        if rc != 0:
            msg = load().slm_batch_last_error(self._h)
            raise SlmError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().slm_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, seed: int = 1, accept_p32: int = P_HALF, max_sweeps: int = 1000,
            max_levels: int = 64, flags: int = 0, stream=None):
        o = Options(seed, accept_p32, max_sweeps, max_levels, flags)
        st = C.c_void_p(int(stream)) if stream is not None else C.c_void_p(0)
        self._check(load().slm_batch_run(self._h, C.byref(o), st))
        return self

    def num_levels(self, g: int) -> int:
        v = C.c_int32()
        self._check(load().slm_batch_num_levels(self._h, g, C.byref(v)))
        return v.value

    def stats(self, g: int, level: int) -> LevelStats:
        s = LevelStats()
        self._check(load().slm_batch_get_stats(self._h, g, level, C.byref(s)))
        return s

    def partition(self, g: int, level: int = -1):
        n = int(self.goff[g + 1] - self.goff[g]) if level == -1 else self.stats(g, level).n
        out = np.zeros(max(n, 1), dtype=np.int32)
        K = C.c_int32()
        self._check(load().slm_batch_get_partition(self._h, g, level, C.c_void_p(out.ctypes.data),
                                                   C.byref(K)))
        return out[:n], K.value

    def modularity(self, g: int) -> float:
        q = C.c_double()
        self._check(load().slm_batch_modularity(self._h, g, C.byref(q)))
        return q.value

    def run_info(self):
        lv = C.c_int32()
        sw = C.c_int64()
        self._check(load().slm_batch_run_info(self._h, C.byref(lv), C.byref(sw)))
        return lv.value, sw.value


def debug_fail_allocation(k: int):
    """The k-th device allocation of the library from now on fails as out of
    memory (k = 0: off); a host-side test hook."""
    load().slm_debug_fail_allocation(int(k))


def footprint(n: int, nnz: int) -> int:
    """Device bytes the request server reserves for a graph of n nodes and nnz entries."""
    return int(load().slm_server_footprint(int(n), int(nnz)))


class Server:
    """Request server (include/slm_server.h): slots with their own streams,
    first-come first-served admission against an HBM budget."""

    def __init__(self, budget_bytes: int, slots: int = 8):
        lib = load()
        self._h = C.c_void_p()
        rc = lib.slm_server_create(int(budget_bytes), int(slots), C.byref(self._h))
        if rc != 0:
            msg = lib.slm_server_last_error(None)
            raise SlmError(rc, msg.decode() if msg else "")

    def _check(self, rc):
        if rc != 0:
            msg = load().slm_server_last_error(self._h)
            raise SlmError(rc, msg.decode() if msg else "")

    def submit(self, row_ptr, col, w=None, *, seed: int = 1, accept_p32: int = P_HALF,
               max_sweeps: int = 1000, max_levels: int = 64, flags: int = 0,
               deadline: float | None = None, directed: bool = False) -> int:
        """Queue one graph (host arrays, copied during the call); returns its
        ticket.  deadline: seconds after submission by which it must end;
        directed: the arrays hold W as out-arcs (slm_server_submit_directed)."""
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        cl = np.ascontiguousarray(col, dtype=np.int32)
        ww = None if w is None else np.ascontiguousarray(w, dtype=np.int32)
        d = GraphDesc(rp.shape[0] - 1, rp.ctypes.data, cl.ctypes.data if cl.size else None,
                      ww.ctypes.data if ww is not None and ww.size else None)
        o = Options(seed, accept_p32, max_sweeps, max_levels, flags)
        t = C.c_uint64()
        if directed:
            self._check(load().slm_server_submit_directed(self._h, C.byref(d), C.byref(o),
                                                          float(deadline or 0.0), C.byref(t)))
        elif deadline is None:
            self._check(load().slm_server_submit(self._h, C.byref(d), C.byref(o), C.byref(t)))
        else:
            self._check(load().slm_server_submit_deadline(self._h, C.byref(d), C.byref(o),
                                                          float(deadline), C.byref(t)))
        return t.value

    def cancel(self, ticket: int):
        """Cancel a queued or running request (it ends FAILED, SLM_ERR_CANCELLED)."""
        self._check(load().slm_server_cancel(self._h, ticket))

    def poll(self, ticket: int) -> int:
        v = C.c_int32()
        self._check(load().slm_server_poll(self._h, ticket, C.byref(v)))
        return v.value

    def wait(self, ticket: int, timeout: float = -1.0) -> bool:
        rc = load().slm_server_wait(self._h, ticket, float(timeout))
        if rc == 8:
            return False
        self._check(rc)
        return True

    def info(self, ticket: int) -> RequestInfo:
        r = RequestInfo()
        self._check(load().slm_server_request_info(self._h, ticket, C.byref(r)))
        return r

    def result(self, ticket: int, release: bool = True):
        """(labels, K, Q) of a finished request; raises SlmError if it failed."""
        n = self.info(ticket).n
        out = np.zeros(max(n, 1), dtype=np.int32)
        K = C.c_int32()
        q = C.c_double()
        self._check(load().slm_server_result(self._h, ticket, C.c_void_p(out.ctypes.data),
                                             C.byref(K), C.byref(q), 1 if release else 0))
        return out[:n], K.value, q.value

    def stats(self) -> ServerStats:
        s = ServerStats()
        self._check(load().slm_server_get_stats(self._h, C.byref(s)))
        return s

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().slm_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Step API on CUDA tensors (one call per step of the method)
# ---------------------------------------------------------------------------
def step_strengths(rp, col, w, stream=None):
    torch = _torch()
    rp, col, w = _dev_i32(rp), _dev_i32(col), _dev_i32(w)
    n = rp.numel() - 1
    s = _empty(n, torch.int32)
    m = C.c_int64()
    _check(load().slm_step_strengths(n, _ptr(rp), _ptr(col), _ptr(w), _ptr(s), C.byref(m),
                                     _stream(stream)))
    return s, m.value


def step_assign(rp, col, w, s, m, stream=None):
    torch = _torch()
    rp, col, w, s = map(_dev_i32, (rp, col, w, s))
    n = rp.numel() - 1
    a = _empty(n, torch.int32)
    _check(load().slm_step_assign(n, _ptr(rp), _ptr(col), _ptr(w), _ptr(s), int(m), _ptr(a),
                                  _stream(stream)))
    return a


def step_components(a, stream=None):
    torch = _torch()
    a = _dev_i32(a)
    root = _empty(a.numel(), torch.int32)
    _check(load().slm_step_components(a.numel(), _ptr(a), _ptr(root), _stream(stream)))
    return root


def step_scan(rp, col, w, s, m, root, stream=None):
    torch = _torch()
    rp, col, w, s, root = map(_dev_i32, (rp, col, w, s, root))
    n = rp.numel() - 1
    best = _empty(n, torch.int32)
    gain = _empty(n, torch.int64)
    g = _empty(n, torch.int64)
    _check(load().slm_step_scan(n, _ptr(rp), _ptr(col), _ptr(w), _ptr(s), int(m), _ptr(root),
                                _ptr(best), _ptr(gain), _ptr(g), _stream(stream)))
    return best, gain, g


def step_branch_gain(rp, col, w, s, m, a, root, best, gain, stream=None):
    torch = _torch()
    rp, col, w, s, a, root, best = map(_dev_i32, (rp, col, w, s, a, root, best))
    gain = gain.to(device="cuda", dtype=torch.int64).contiguous()
    if gain.numel() == 0:
        gain = torch.zeros(1, dtype=torch.int64, device="cuda")
    n = rp.numel() - 1
    bg = _empty(n, torch.int64)
    _check(load().slm_step_branch_gain(n, _ptr(rp), _ptr(col), _ptr(w), _ptr(s), int(m), _ptr(a),
                                       _ptr(root), _ptr(best), _ptr(gain), _ptr(bg),
                                       _stream(stream)))
    return bg


def step_maximal(rp, col, w, s, m, a, root, seed, accept_p32, level, sweep, stream=None):
    rp, col, w, s, root = map(_dev_i32, (rp, col, w, s, root))
    a = _dev_i32(a).clone()
    n = rp.numel() - 1
    counts = np.zeros(3, dtype=np.int64)
    _check(load().slm_step_maximal(n, _ptr(rp), _ptr(col), _ptr(w), _ptr(s), int(m), _ptr(a),
                                   _ptr(root), int(seed), int(accept_p32), int(level), int(sweep),
                                   C.c_void_p(counts.ctypes.data), _stream(stream)))
    return a, counts


def step_positive(rp, col, w, s, m, a, stream=None):
    torch = _torch()
    rp, col, w, s = map(_dev_i32, (rp, col, w, s))
    a = _dev_i32(a).clone()
    n = rp.numel() - 1
    root = _empty(n, torch.int32)
    splits = np.zeros(1, dtype=np.int64)
    _check(load().slm_step_positive(n, _ptr(rp), _ptr(col), _ptr(w), _ptr(s), int(m), _ptr(a),
                                    _ptr(root), C.c_void_p(splits.ctypes.data), _stream(stream)))
    return a, root, int(splits[0])


def step_compact(root, stream=None):
    torch = _torch()
    root = _dev_i32(root)
    idv = _empty(root.numel(), torch.int32)
    K = C.c_int32()
    _check(load().slm_step_compact(root.numel(), _ptr(root), _ptr(idv), C.byref(K),
                                   _stream(stream)))
    return idv, K.value


def step_aggregate(rp, col, w, idv, K, stream=None):
    torch = _torch()
    rp, col, w, idv = map(_dev_i32, (rp, col, w, idv))
    n = rp.numel() - 1
    rp2 = _empty(K + 1, torch.int32)
    col2 = _empty(max(col.numel(), 1), torch.int32)
    w2 = _empty(max(col.numel(), 1), torch.int32)
    nnz = C.c_int32()
    _check(load().slm_step_aggregate(n, _ptr(rp), _ptr(col), _ptr(w), _ptr(idv), int(K),
                                     _ptr(rp2), _ptr(col2), _ptr(w2), C.byref(nnz),
                                     _stream(stream)))
    return rp2, col2[: nnz.value], w2[: nnz.value]


def step_modularity_noalloc(rp, col, w, labels, stream=None):
    """Modularity through the entry point that allocates no device memory;
    returns (q, num) read back from the device outputs."""
    torch = _torch()
    rp, col, w, labels = map(_dev_i32, (rp, col, w, labels))
    n = rp.numel() - 1
    num = torch.zeros(1, dtype=torch.int64, device="cuda")
    q = torch.zeros(1, dtype=torch.float64, device="cuda")
    _check(load().slm_step_modularity_noalloc(n, _ptr(rp), _ptr(col), _ptr(w), _ptr(labels),
                                              _ptr(num), _ptr(q), _stream(stream)))
    return float(q.item()), int(num.item())


def step_modularity(rp, col, w, labels, stream=None):
    rp, col, w, labels = map(_dev_i32, (rp, col, w, labels))
    n = rp.numel() - 1
    q = C.c_double()
    num = C.c_int64()
    _check(load().slm_step_modularity(n, _ptr(rp), _ptr(col), _ptr(w), _ptr(labels), C.byref(q),
                                      C.byref(num), _stream(stream)))
    return q.value, num.value
