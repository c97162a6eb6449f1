"""Autotuner of the MAXIMAL scan's launch shapes.

The scan runs one kernel shape per fine degree class (a thread per node,
lane groups, blocks of several sizes, hub chunks).  Which of two shapes each
class uses -- and with it where the boundaries between the thread, lane-group
and block kernels fall --, how many blocks each shape may launch per SM, and
whether the classes run side by side on four streams or one after another,
decide how well they share the GPU for a given degree distribution.  None of
it changes a result.

``autotune_scan`` times the scan (``slm_step_scan``: degree buckets,
community totals and the scan kernels) on a graph's own level-0 state --
after ASSIGN and POSITIVE -- under candidate tunings, by coordinate descent
from the current tuning: each field in turn takes the value that makes the
scan fastest; then each class's shape bit in turn.  Every candidate's outputs (best community, gain, local gain)
are compared with the starting tuning's and must be identical.  The winner
is applied process-wide (``slm_set_scan_tuning``) and remembered per graph
shape (node count, entry count and degree histogram) for the rest of the
process.
"""
from __future__ import annotations

import numpy as np

from . import (get_scan_tuning, set_scan_tuning, step_assign, step_positive, step_scan,
               step_strengths)

# values tried per field; the first run starts from the current tuning
SPACE = {
    "streams": [4, 1],
    "blocks_large": [1, 2, 3],
    "blocks_mid": [2, 4, 6],
    "blocks_small": [4, 6, 8],
    "blocks_warp": [4, 6, 8, 16],
    "blocks_hub": [4, 8, 16],
    "blocks_group": [8, 16, 32],
}
NUM_CLASSES = 11  # fine degree classes with a choice of shape (bit k-1 of shape_alt)

_cache: dict = {}


def shape_key(row_ptr) -> tuple:
    """Node count, entry count and the log2 degree histogram of a CSR."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    deg = np.diff(rp)
    hist = np.bincount(np.ceil(np.log2(np.maximum(deg, 1))).astype(np.int64), minlength=24)
    return (int(rp.shape[0] - 1), int(rp[-1]), tuple(int(x) for x in hist[:24]))


def _time_scan(args, reps: int, torch) -> float:
    """Median milliseconds of one slm_step_scan call over `reps` calls."""
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        step_scan(*args)
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def autotune_scan(row_ptr, col, w, reps: int = 5, apply: bool = True, use_cache: bool = True):
    """Pick the scan tuning for this graph; returns (tuning, report).

    row_ptr, col, w: the graph's CSR (host arrays or CUDA tensors).  The
    report lists every candidate's median time in milliseconds."""
    import torch

    rp_h = row_ptr.cpu().numpy() if hasattr(row_ptr, "cpu") else np.asarray(row_ptr)
    key = shape_key(rp_h)
    if use_cache and key in _cache:
        best = dict(_cache[key])
        if apply:
            set_scan_tuning(**best)
        return best, {"cached": True}
    dev = torch.device("cuda", torch.cuda.current_device())
    rp, cl, ww = (torch.as_tensor(np.asarray(x) if not hasattr(x, "cpu") else x,
                                  dtype=torch.int32).to(dev) for x in (row_ptr, col, w))
    s, m = step_strengths(rp, cl, ww)
    a = step_assign(rp, cl, ww, s, m)
    a, root, _ = step_positive(rp, cl, ww, s, m, a)
    args = (rp, cl, ww, s, m, root)
    start = get_scan_tuning()
    ref = [t.cpu() for t in step_scan(*args)]
    _time_scan(args, 2, torch)  # warm-up
    best = dict(start)
    best_ms = _time_scan(args, reps, torch)
    report = {"start": dict(start), "start_ms": best_ms, "tried": []}
    trials = [(f, v) for f, values in SPACE.items() for v in values]
    trials += [("shape_alt", bit) for bit in range(NUM_CLASSES)]
    for field, v in trials:
        cand = dict(best)
        if field == "shape_alt":
            cand[field] = best[field] ^ (1 << v)
        elif v == best[field]:
            continue
        else:
            cand[field] = v
        set_scan_tuning(**cand)
        out = [t.cpu() for t in step_scan(*args)]
        for x, y in zip(out, ref):
            if not torch.equal(x, y):
                set_scan_tuning(**start)
                raise RuntimeError(f"scan outputs changed under tuning {cand}")
        ms = _time_scan(args, reps, torch)
        report["tried"].append((cand, ms))
        if ms < best_ms:
            best, best_ms = cand, ms
        set_scan_tuning(**best)
    report["best"] = dict(best)
    report["best_ms"] = best_ms
    _cache[key] = dict(best)
    set_scan_tuning(**(best if apply else start))
    return best, report
