"""Synchronised Louvain against classical sequential-move Louvain (the
comparison the paper's conclusion, Section 6, proposes), both as the oracle
runs them, on the seeded workloads: final modularity, communities, agreement
with the planted partition (NMI) where there is one, levels, sweeps or passes,
and single-thread CPU time.

    python oracle/compare_louvain.py

Test infrastructure like the rest of oracle/: it calls only the oracle and
the graph generators.  The synchronised runs here are the same partitions the
GPU library produces (checked by the parity tests on these graphs).
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402
import oracle as O  # noqa: E402


def nmi(a, b) -> float:
    """Normalised mutual information (arithmetic-mean normalisation)."""
    a = np.unique(np.asarray(a), return_inverse=True)[1].astype(np.int64)
    b = np.unique(np.asarray(b), return_inverse=True)[1].astype(np.int64)
    n, kb = a.shape[0], int(b.max()) + 1
    keys, cnt = np.unique(a * kb + b, return_counts=True)
    pa, pb, pij = np.bincount(a) / n, np.bincount(b) / n, cnt / n
    ha, hb = -(pa * np.log(pa)).sum(), -(pb * np.log(pb)).sum()
    mi = (pij * np.log(pij / (pa[keys // kb] * pb[keys % kb]))).sum()
    return float(2 * mi / (ha + hb)) if ha + hb > 0 else 1.0


def workloads():
    out = []
    for mt, mw in [(0.2, 0.1), (0.5, 0.4), (0.8, 0.7)]:
        g, comm = gg.lfr_weighted(10000, mt, mw)
        out.append((f"weighted LFR 10^4 ({mt},{mw})", g, comm))
    sbm = gg.sbm_planted()
    out.append(("planted partition 10^4 (20x500)", sbm, np.repeat(np.arange(20), 500)))
    out.append(("R-MAT scale 14", gg.rmat(scale=14, seed=2), None))
    return out


def main():
    rows = []
    for name, g, planted in workloads():
        t0 = time.perf_counter()
        r = O.slm(g, seed=1, P=O.P_HALF)
        t_slm = time.perf_counter() - t0
        t0 = time.perf_counter()
        c = O.louvain(g)
        t_lv = time.perf_counter() - t0
        row = [name, f"{g.n:,} / {g.nnz:,}"]
        for run, t in ((r, t_slm), (c, t_lv)):
            K = int(run.final.max()) + 1 if g.n else 0
            sweeps = sum(st[0] for st in run.stats) + run.top[1]
            row += [f"{O.modularity(g, run.final):.4f}", str(K),
                    "-" if planted is None else f"{nmi(run.final, planted):.3f}",
                    f"{run.num_levels} / {sweeps}", f"{t:.2f}"]
        rows.append(row)
        print(" | ".join(row), flush=True)
    head = ["graph", "n / entries", "SLM Q", "SLM K", "SLM NMI", "SLM levels / sweeps", "SLM s",
            "Louvain Q", "Louvain K", "Louvain NMI", "Louvain levels / passes", "Louvain s"]
    print()
    print("| " + " | ".join(head) + " |")
    print("|" + "---|" * len(head))
    for row in rows:
        print("| " + " | ".join(row) + " |")


if __name__ == "__main__":
    main()
