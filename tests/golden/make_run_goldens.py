"""Write the oracle's whole-run results on the benchmark-sized graphs.

Usage: python tests/golden/make_run_goldens.py [case ...]   (all cases by default)

Each case regenerates a seeded graph with ``graphgen`` and runs the CPU oracle
on it, single-threaded: ``oracle.slm`` (Algorithm 1 with ASSIGN, POSITIVE and
MAXIMAL as the oracle restates them), ``oracle.directed_slm`` (the same on a
directed graph), or for the comparison method ``oracle.louvain_colour``
(colour-synchronous Louvain); nothing here touches the CUDA library.
The result goes to ``tests/golden/run_<case>.json``:

  graph    n, nnz, m_w and SHA-256 digests of row_ptr, col and w (int32,
           little-endian), so a test can tell a changed generator from a
           changed run;
  levels   per recorded level: n, K, the SHA-256 of its int32 community ids
           and the level stats (sweeps, stop reason, moves, splits,
           candidates, entries scanned);
  final    SHA-256 of the composed labels on the input nodes and their K;
  trace    every sweep's row (level, sweep, candidates, positive branch
           gains, accepted, splits);
  top      stop reason and sweeps of the last, unrecorded level, and the
           level-limit flag;
  q        the oracle's modularity of the final partition (float.hex).

The oracle needs minutes per case; the seconds each case took are stored as
``oracle_seconds`` (wall clock on the machine that wrote the file).
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402
import oracle as O  # noqa: E402


def _rmat_s20():
    return gg.cached("rmat_s20_seed2", gg.rmat, scale=20, seed=2)


def _lfr_4m():
    return gg.cached("lfr_style_default", lambda: gg.lfr_style()[0])


def _lfr_256k():
    return gg.cached("lfr_style_n262144", lambda: gg.lfr_style(n=262144)[0])


# case name -> (graph, run options, description[, oracle method])
CASES = {
    "rmat_s20": (_rmat_s20, dict(seed=1, P=O.P_HALF),
                 "R-MAT scale 20 (seed 2), complete run, acceptance seed 1, p = 1/2"),
    "lfr_4m_bounded": (_lfr_4m, dict(seed=1, P=O.P_HALF, max_sweeps=2, max_levels=3),
                       "LFR-style 4,194,304 nodes (seed 3), at most 2 sweeps per level and 3 levels"),
    "lfr_4m_level0": (_lfr_4m, dict(seed=1, P=O.P_HALF, max_sweeps=2, max_levels=1),
                      "LFR-style 4,194,304 nodes (seed 3), level 0 only, at most 2 sweeps"),
    "lfr_4m_level0": (_lfr_4m, dict(seed=1, P=O.P_HALF, max_sweeps=2, max_levels=1),
                      "LFR-style 4,194,304 nodes (seed 3), level 0 only, at most 2 sweeps"),
    "lfr_256k_bounded": (_lfr_256k, dict(seed=1, P=O.P_HALF, max_sweeps=3),
                         "LFR-style 262,144 nodes (seed 3), at most 3 sweeps per level, every level"),
    "lfr_directed_1e4_high_mixing": (lambda: gg.lfr_directed(10000, 0.8, 0.7)[0], dict(seed=3, P=O.P_HALF),
                                     "directed weighted LFR-style, 10,000 nodes, (mu_t, mu_w) = (0.8, 0.7), "
                                     "complete run (directed Q_w)", "directed_slm"),
    "louvain_rmat_s20": (_rmat_s20, dict(seed=1),
                         "colour-synchronous Louvain on R-MAT scale 20 (seed 2), colouring seed 1, "
                         "complete run", "louvain_colour"),
}


def sha(x) -> str:
    return hashlib.sha256(np.ascontiguousarray(x, dtype="<i4").tobytes()).hexdigest()


def fingerprint(g) -> dict:
    m = int(np.asarray(g.w, dtype=np.int64).sum())
    return {"n": int(g.n), "nnz": int(g.nnz), "m_w": m, "row_ptr": sha(g.row_ptr),
            "col": sha(g.col), "w": sha(g.w)}


def make(case: str) -> dict:
    gen, opts, desc = CASES[case][:3]
    method = CASES[case][3] if len(CASES[case]) > 3 else "slm"
    g = gen()
    t0 = time.time()
    r = getattr(O, method)(g, **opts)
    dt = time.time() - t0
    q = (O.directed_modularity if method == "directed_slm" else O.modularity)(g, r.final)
    levels = []
    for (ids, K), st in zip(r.levels, r.stats):
        levels.append({"n": int(ids.shape[0]), "K": int(K), "ids": sha(ids), "stats": list(st)})
    out = {
        "case": case,
        "description": desc,
        "method": method,
        "options": {k: int(v) for k, v in opts.items()},
        "graph": fingerprint(g),
        "levels": levels,
        "final": {"labels": sha(r.final), "K": int(r.final.max()) + 1 if g.n else 0},
        "trace": r.trace.tolist(),
        "top": list(r.top),
        "q": float(q).hex(),
        "oracle_seconds": round(dt, 1),
    }
    with open(os.path.join(HERE, f"run_{case}.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    return out


if __name__ == "__main__":
    for c in sys.argv[1:] or list(CASES):
        o = make(c)
        print(c, "levels", len(o["levels"]), "sweeps", len(o["trace"]), "oracle s", o["oracle_seconds"],
              flush=True)
