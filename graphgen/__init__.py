"""Seeded synthetic graph generators (inputs only).

This module produces the symmetric integer-weighted CSR graphs that both the
CUDA path and the CPU oracle consume.  It holds none of the method's
arithmetic: no gain, no modularity, no assignment.  Every random number is
drawn from a counter-based generator (the splitmix64 finaliser of Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014)
keyed by (seed, stream, counter), so a graph is a pure function of its
parameters on every machine and numpy version.

CSR conventions (shared by the library and the oracle):
  * ``row_ptr`` int32[n+1], ``col`` int32[nnz], ``w`` int32[nnz];
  * columns of every row sorted ascending and unique;
  * W symmetric, w > 0; a self-loop W_uu is stored once in row u.

The paper's experiments use LFR benchmark graphs (Section 5.1, Table 1); the
generators here are seeded stand-ins shaped like the workloads the library is
measured on (planted partitions, R-MAT, an LFR-style power-law graph, a forest
of many small planted-partition graphs and a Poisson stream of R-MAT
requests).
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass

import numpy as np

__all__ = [
    "CSR", "mix64", "uniform01", "uniform_int", "from_edges", "sbm_planted",
    "rmat", "lfr_style", "forest_sbm_params", "forest_sbm_graph", "served_stream",
    "star", "path", "ring_of_cliques", "two_cliques", "random_small",
    "isolated_and_loops", "cached",
]

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)


@dataclass
class CSR:
    n: int
    row_ptr: np.ndarray  # int32[n+1]
    col: np.ndarray      # int32[nnz]
    w: np.ndarray        # int32[nnz]

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def arrays(self):
        return self.row_ptr, self.col, self.w


def mix64(z: np.ndarray) -> np.ndarray:
    """splitmix64 output function applied elementwise to uint64 values."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
    return z ^ (z >> np.uint64(31))


def _draw_u64(seed, stream: int, idx) -> np.ndarray:
    """64 random bits for (seed, stream, counter); seed may be an array of the
    same shape as idx (one seed per draw)."""
    idx = np.asarray(idx, dtype=np.uint64)
    if np.ndim(seed) == 0:
        key = np.uint64(int(seed) & 0xFFFFFFFFFFFFFFFF)
    else:
        key = np.asarray(seed, dtype=np.uint64)
    with np.errstate(over="ignore"):
        s = mix64(np.uint64(stream & 0xFFFFFFFFFFFFFFFF) ^ key)
        return mix64(idx ^ s)


def uniform01(seed, stream: int, idx) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    u = _draw_u64(seed, stream, idx) >> np.uint64(11)
    return u.astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_int(seed, stream: int, idx, lo: int, hi: int) -> np.ndarray:
    """Integers uniform in [lo, hi] (inclusive) by a multiply-shift on 32 bits."""
    span = np.uint64(hi - lo + 1)
    u = _draw_u64(seed, stream, idx) >> np.uint64(32)
    return (lo + ((u * span) >> np.uint64(32)).astype(np.int64)).astype(np.int64)


def from_edges(n: int, u, v, w=None, *, unit: bool = False) -> CSR:
    """Canonical symmetric CSR from undirected draws.

    A draw (u, v, w) with u != v adds w to W_uv and to W_vu; a draw (u, u, w)
    adds w to W_uu once.  Duplicates are merged by summing, or collapsed to a
    single unit edge when ``unit`` is set.
    """
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    if w is None:
        w = np.ones(u.shape[0], dtype=np.int64)
    w = np.asarray(w, dtype=np.int64)
    off = u != v
    src = np.concatenate([u, v[off]])
    dst = np.concatenate([v, u[off]])
    ww = np.concatenate([w, w[off]])
    key = src * np.int64(n) + dst
    order = np.argsort(key)
    key = key[order]
    ww = ww[order]
    if key.shape[0]:
        first = np.ones(key.shape[0], dtype=bool)
        first[1:] = key[1:] != key[:-1]
        starts = np.flatnonzero(first)
        ukey = key[starts]
        if unit:
            uw = np.ones(ukey.shape[0], dtype=np.int64)
        else:
            uw = np.add.reduceat(ww, starts)
    else:
        ukey = key
        uw = ww
    rows = (ukey // n).astype(np.int64)
    cols = (ukey % n).astype(np.int64)
    counts = np.bincount(rows, minlength=n) if n else np.zeros(0, np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2**31 or (uw.shape[0] and uw.max() >= 2**31):
        raise ValueError("graph too large for int32 CSR")
    return CSR(n, row_ptr.astype(np.int32), cols.astype(np.int32), uw.astype(np.int32))


# ---------------------------------------------------------------------------
# Planted partition (stochastic block model), Bernoulli per node pair.
# ---------------------------------------------------------------------------
def sbm_planted(n_blocks: int = 20, block_size: int = 500, p_in: float = 16 / 499,
                p_out: float = 4 / 9500, seed: int = 1) -> CSR:
    """Undirected planted partition with unit weights; pair (i<j) is an edge
    with probability p_in inside a block and p_out across blocks."""
    n = n_blocks * block_size
    us, vs = [], []
    block = np.arange(n) // block_size
    for i in range(n - 1):
        j = np.arange(i + 1, n, dtype=np.int64)
        r = uniform01(seed, 0, np.int64(i) * n + j)
        p = np.where(block[j] == block[i], p_in, p_out)
        hit = j[r < p]
        if hit.shape[0]:
            us.append(np.full(hit.shape[0], i, dtype=np.int64))
            vs.append(hit)
    u = np.concatenate(us) if us else np.zeros(0, np.int64)
    v = np.concatenate(vs) if vs else np.zeros(0, np.int64)
    return from_edges(n, u, v)


# ---------------------------------------------------------------------------
# R-MAT (Chakrabarti, Zhan, Faloutsos 2004).
# ---------------------------------------------------------------------------
def rmat(scale: int = 20, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, wmin: int = 1, wmax: int = 8, seed: int = 2,
         n: int | None = None, draws: int | None = None, permute: bool = True) -> CSR:
    """R-MAT graph: ``draws`` endpoint pairs chosen by recursive quadrant
    descent with probabilities (a, b, c, 1-a-b-c) quantised to 1/65536, integer weights uniform in
    [wmin, wmax], vertex ids permuted by a seeded random relabelling, self-loops
    and duplicates merged by summing.  When ``n`` is below 2**scale, draws with
    an endpoint >= n are redrawn (with a fresh counter) until both fit."""
    N = 1 << scale
    if n is None:
        n = N
    if draws is None:
        draws = edge_factor * N
    idx = np.arange(draws, dtype=np.int64)
    u = np.zeros(draws, dtype=np.int64)
    v = np.zeros(draws, dtype=np.int64)
    todo = idx
    attempt = 0
    while todo.shape[0]:
        uu = np.zeros(todo.shape[0], dtype=np.int64)
        vv = np.zeros(todo.shape[0], dtype=np.int64)
        ctr = todo + np.int64(attempt) * np.int64(draws)
        # one 64-bit draw feeds four levels with 16-bit quadrant probabilities
        ta, tab, tabc = (np.uint64(int(round(x * 65536))) for x in (a, a + b, a + b + c))
        for lvl0 in range(0, scale, 4):
            bits = _draw_u64(seed, 1 + lvl0 // 4, ctr)
            for k in range(min(4, scale - lvl0)):
                r = (bits >> np.uint64(16 * k)) & np.uint64(0xFFFF)
                bu = (r >= tab).astype(np.int64)
                bv = (((r >= ta) & (r < tab)) | (r >= tabc)).astype(np.int64)
                uu = (uu << 1) | bu
                vv = (vv << 1) | bv
        u[todo] = uu
        v[todo] = vv
        bad = (uu >= n) | (vv >= n)
        todo = todo[bad]
        attempt += 1
    w = uniform_int(seed, 100, idx, wmin, wmax)
    if permute:
        keys = _draw_u64(seed, 101, np.arange(n, dtype=np.int64))
        order = np.argsort(keys, kind="stable")
        relabel = np.empty(n, dtype=np.int64)
        relabel[order] = np.arange(n, dtype=np.int64)
        u = relabel[u]
        v = relabel[v]
    return from_edges(n, u, v, w)


# ---------------------------------------------------------------------------
# LFR-style power-law graph with planted communities (after Lancichinetti,
# Fortunato, Radicchi 2008), wired by a configuration model.
# ---------------------------------------------------------------------------
def _powerlaw_int(seed, stream, count, expo, lo, hi):
    """Integers in [lo, hi] with P(k) ~ k^-expo, by inverse transform of the
    continuous law on [lo, hi+1) followed by flooring."""
    r = uniform01(seed, stream, np.arange(count, dtype=np.int64))
    if expo == 1.0:  # log-uniform
        x = float(lo) * (float(hi + 1) / float(lo)) ** r
        return np.clip(np.floor(x).astype(np.int64), lo, hi)
    g = 1.0 - expo
    a_ = float(lo) ** g
    b_ = float(hi + 1) ** g
    x = (a_ + r * (b_ - a_)) ** (1.0 / g)
    return np.clip(np.floor(x).astype(np.int64), lo, hi)


def _powerlaw_mean(expo, lo, hi):
    k = np.arange(lo, hi + 1, dtype=np.float64)
    # continuous law on [k, k+1) integrated, matching _powerlaw_int
    g = 1.0 - expo
    cdf = (lambda x: np.log(x)) if expo == 1.0 else (lambda x: x ** g)  # noqa: E731
    p = (cdf(k + 1) - cdf(k)) / (cdf(float(hi + 1)) - cdf(float(lo)))
    return float((p * k).sum())


def lfr_style(n: int = 4194304, tau1: float = 2.5, kavg: float = 20.0, kmax: int = 5000,
              tau2: float = 1.5, cmin: int = 50, cmax: int = 50000, mu: float = 0.3,
              seed: int = 3) -> tuple[CSR, np.ndarray]:
    """LFR-style benchmark graph; returns (CSR, planted community of each node).

    Degrees follow a power law (exponent tau1, maximum kmax) whose minimum is
    chosen so that the mean is kavg; community sizes follow a power law
    (exponent tau2) in [cmin, cmax].  Each node sends round((1-mu)*d) stubs
    inside its community (capped at community size - 1) and the rest outside.
    Stubs are paired uniformly at random inside each community and across the
    whole graph; self-loops are dropped and duplicate pairs collapse to one
    unit-weight edge."""
    u, v, _, comm = _lfr_wiring(n, tau1, kavg, kmax, tau2, cmin, cmax, mu, seed)
    return from_edges(n, u, v, unit=True), comm


def lfr_weighted(n: int, mu_t: float, mu_w: float, kavg: float = 50.0, kmax: int = 100,
                 tau1: float = 2.0, tau2: float = 1.0, cmin: int = 100, cmax: int = 1000,
                 wbar: int = 8, seed: int = 5) -> tuple[CSR, np.ndarray]:
    """Weighted LFR-style graph with topology mixing mu_t and weight mixing
    mu_w (the benchmark family of the paper's experiments: mean degree 50,
    maximum degree 100, (mu_t, mu_w) in {(0.2, 0.1), (0.5, 0.4), (0.8, 0.7)});
    returns (CSR, planted community of each node).

    The wiring is lfr_style's.  An internal edge draws its weight uniformly
    from [1, 2*t_in - 1] and an external one from [1, 2*t_out - 1], with
    t_in = round(wbar*(1 - mu_w)/(1 - mu_t)) and t_out = round(wbar*mu_w/mu_t)
    (at least 1), so that a node of degree d has expected strength about
    d*wbar of which about a fraction mu_w lies on external edges.  One draw
    gives both directions of an edge; duplicate pairs sum their weights."""
    u, v, internal, comm = _lfr_wiring(n, tau1, kavg, kmax, tau2, cmin, cmax, mu_t, seed)
    t_in = max(1, int(round(wbar * (1.0 - mu_w) / (1.0 - mu_t))))
    t_out = max(1, int(round(wbar * mu_w / mu_t)))
    idx = np.arange(u.shape[0], dtype=np.int64)
    w = np.where(internal, uniform_int(seed, 5, idx, 1, 2 * t_in - 1),
                 uniform_int(seed, 6, idx, 1, 2 * t_out - 1))
    return from_edges(n, u, v, w), comm


def lfr_directed(n: int, mu_t: float, mu_w: float, recip: float = 0.3, **kw) -> tuple[CSR, np.ndarray]:
    """Directed weighted LFR-style graph: the wiring and weights of
    lfr_weighted, each stub pair becoming an arc in a random direction, and
    with probability `recip` also the reverse arc (its own weight draw).
    Returns (directed CSR, planted community of each node)."""
    args = dict(kavg=50.0, kmax=100, tau1=2.0, tau2=1.0, cmin=100, cmax=1000, wbar=8, seed=5)
    args.update(kw)
    seed, wbar = args.pop("seed"), args.pop("wbar")
    u, v, internal, comm = _lfr_wiring(n, args["tau1"], args["kavg"], args["kmax"], args["tau2"],
                                       args["cmin"], args["cmax"], mu_t, seed)
    t_in = max(1, int(round(wbar * (1.0 - mu_w) / (1.0 - mu_t))))
    t_out = max(1, int(round(wbar * mu_w / mu_t)))
    idx = np.arange(u.shape[0], dtype=np.int64)
    flip = uniform01(seed, 7, idx) < 0.5
    a, b = np.where(flip, v, u), np.where(flip, u, v)
    back = uniform01(seed, 8, idx) < recip
    w1 = np.where(internal, uniform_int(seed, 5, idx, 1, 2 * t_in - 1),
                  uniform_int(seed, 6, idx, 1, 2 * t_out - 1))
    w2 = np.where(internal, uniform_int(seed, 9, idx, 1, 2 * t_in - 1),
                  uniform_int(seed, 10, idx, 1, 2 * t_out - 1))
    return (directed_from_edges(n, np.concatenate([a, b[back]]), np.concatenate([b, a[back]]),
                                np.concatenate([w1, w2[back]])), comm)


def _lfr_wiring(n, tau1, kavg, kmax, tau2, cmin, cmax, mu, seed):
    """The stub pairs of an LFR-style graph without self-loops: (u, v, drawn
    inside a community, planted community of each node)."""
    # minimum degree giving the requested mean
    kmin = 1
    for k0 in range(1, kmax):
        if _powerlaw_mean(tau1, k0, kmax) >= kavg:
            kmin = k0
            break
    deg = _powerlaw_int(seed, 1, n, tau1, kmin, kmax)
    # community sizes until they cover n
    sizes = []
    total = 0
    chunk = 0
    while total < n:
        s = _powerlaw_int(seed, 1000 + chunk, 4096, tau2, cmin, cmax)
        for x in s.tolist():
            if total >= n:
                break
            sizes.append(x)
            total += x
        chunk += 1
    excess = total - n
    sizes[-1] -= excess
    if sizes[-1] < cmin and len(sizes) > 1:
        sizes[-2] += sizes[-1]
        sizes.pop()
    sizes = np.array(sizes, dtype=np.int64)
    # internal stubs per node
    k_in = np.rint((1.0 - mu) * deg).astype(np.int64)
    # place high internal degree nodes in large communities: sort both
    node_order = np.lexsort((_draw_u64(seed, 2, np.arange(n)), -k_in))
    comm_order = np.argsort(-sizes, kind="stable")
    comm_of_slot = np.repeat(comm_order, sizes[comm_order])
    comm = np.empty(n, dtype=np.int64)
    comm[node_order] = comm_of_slot
    k_in = np.minimum(k_in, sizes[comm] - 1)
    k_out = deg - k_in
    # internal wiring: stubs sorted by (community, random key), paired in order
    stub_node = np.repeat(np.arange(n, dtype=np.int64), k_in)
    stub_comm = comm[stub_node]
    key = _draw_u64(seed, 3, np.arange(stub_node.shape[0], dtype=np.int64))
    order = np.lexsort((key, stub_comm))
    stub_node = stub_node[order]
    stub_comm = stub_comm[order]
    # pair consecutive stubs of the same community
    cnt = np.bincount(stub_comm, minlength=sizes.shape[0])
    start = np.zeros(sizes.shape[0] + 1, dtype=np.int64)
    np.cumsum(cnt, out=start[1:])
    pos_in = np.arange(stub_node.shape[0], dtype=np.int64) - start[stub_comm]
    usable = pos_in < (cnt[stub_comm] // 2) * 2
    sn = stub_node[usable]
    ui, vi = sn[0::2], sn[1::2]
    # external wiring
    ext = np.repeat(np.arange(n, dtype=np.int64), k_out)
    key = _draw_u64(seed, 4, np.arange(ext.shape[0], dtype=np.int64))
    ext = ext[np.argsort(key, kind="stable")]
    if ext.shape[0] % 2:
        ext = ext[:-1]
    ue, ve = ext[0::2], ext[1::2]
    u = np.concatenate([ui, ue])
    v = np.concatenate([vi, ve])
    internal = np.concatenate([np.ones(ui.shape[0], bool), np.zeros(ue.shape[0], bool)])
    keep = u != v
    return u[keep], v[keep], internal[keep], comm


# ---------------------------------------------------------------------------
# Forest of planted-partition graphs (the batched workload).
# ---------------------------------------------------------------------------
def forest_sbm_params(num_graphs: int = 4096, nmin: int = 100, nmax: int = 50000,
                      bmin: int = 4, bmax: int = 64, seed_base: int = 1000):
    """Per-graph (n, blocks, seed) of the forest: n log-uniform in [nmin, nmax]
    and blocks uniform in {bmin..bmax}, drawn from the graph's own seed."""
    out = []
    for g in range(num_graphs):
        sd = seed_base + g
        r = float(uniform01(sd, 0, np.array([0]))[0])
        n = int(round(math.exp(math.log(nmin) + r * (math.log(nmax) - math.log(nmin)))))
        nb = int(uniform_int(sd, 1, np.array([0]), bmin, bmax)[0])
        out.append((n, min(nb, n), sd))
    return out


def forest_sbm_graph(n: int, blocks: int, seed: int, deg_in: float = 12.0,
                     deg_out: float = 3.0, wmin: int = 1, wmax: int = 4) -> CSR:
    """Planted partition with ``blocks`` contiguous near-equal blocks: round(n*deg_in/2)
    intra-block and round(n*deg_out/2) inter-block draws with uniform endpoints,
    integer weights uniform in [wmin, wmax]; self-draws dropped, duplicates summed."""
    block_start = (np.arange(blocks + 1, dtype=np.int64) * n) // blocks
    block_of = np.repeat(np.arange(blocks, dtype=np.int64), np.diff(block_start))
    m_in = int(round(n * deg_in / 2))
    m_out = int(round(n * deg_out / 2)) if blocks > 1 else 0
    i_in = np.arange(m_in, dtype=np.int64)
    u1 = (uniform01(seed, 10, i_in) * n).astype(np.int64)
    b1 = block_of[u1]
    bs = block_start[b1]
    bl = block_start[b1 + 1] - bs
    v1 = bs + (uniform01(seed, 11, i_in) * bl).astype(np.int64)
    i_out = np.arange(m_out, dtype=np.int64)
    u2 = (uniform01(seed, 12, i_out) * n).astype(np.int64)
    b2 = block_of[u2]
    bs2 = block_start[b2]
    bl2 = block_start[b2 + 1] - bs2
    r = (uniform01(seed, 13, i_out) * (n - bl2)).astype(np.int64)
    v2 = np.where(r >= bs2, r + bl2, r)
    u = np.concatenate([u1, u2])
    v = np.concatenate([v1, v2])
    w = uniform_int(seed, 14, np.arange(u.shape[0], dtype=np.int64), wmin, wmax)
    keep = u != v
    return from_edges(n, u[keep], v[keep], w[keep])


def forest_sbm(params, deg_in: float = 12.0, deg_out: float = 3.0, wmin: int = 1, wmax: int = 4,
               chunk: int = 256, workers: int = 0):
    """All graphs of forest_sbm_params packed as one block-diagonal CSR:
    returns (graph_off, row_ptr, col, w, seeds).  Graph g is exactly
    forest_sbm_graph(n_g, blocks_g, seed_g) shifted by graph_off[g].  Graphs
    are drawn `chunk` at a time with vectorised draws, in `workers` spawned
    processes when workers > 1 (the result does not depend on it)."""
    jobs = [(params[k:k + chunk], deg_in, deg_out, wmin, wmax)
            for k in range(0, len(params), chunk)]
    if workers and workers > 1 and len(jobs) > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(workers, len(jobs))) as pool:
            parts = pool.starmap(_forest_sbm_chunk, jobs)
    else:
        parts = [_forest_sbm_chunk(*j) for j in jobs]
    G = len(params)
    goff = np.zeros(G + 1, dtype=np.int64)
    rps, cols, ws = [], [], []
    nbase, ebase, g0 = 0, 0, 0
    for (pg, prp, pcol, pw, _) in parts:
        k = pg.shape[0] - 1
        goff[g0 + 1: g0 + k + 1] = pg[1:].astype(np.int64) + nbase
        rps.append(prp[1:].astype(np.int64) + ebase)
        cols.append(pcol.astype(np.int64) + nbase)
        ws.append(pw)
        nbase += int(pg[-1])
        ebase += int(prp[-1])
        g0 += k
    if ebase >= 2**31:
        raise ValueError("forest too large for int32 CSR")
    rp = np.concatenate([np.zeros(1, np.int64)] + rps).astype(np.int32)
    col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    w = np.concatenate(ws).astype(np.int32) if ws else np.zeros(0, np.int32)
    sds = np.array([p[2] for p in params], dtype=np.uint64)
    return goff.astype(np.int32), rp, col, w, sds


def _forest_sbm_chunk(params, deg_in, deg_out, wmin, wmax):
    G = len(params)
    ns = np.array([p[0] for p in params], dtype=np.int64)
    bs = np.array([p[1] for p in params], dtype=np.int64)
    sds = np.array([p[2] for p in params], dtype=np.uint64)
    goff = np.zeros(G + 1, dtype=np.int64)
    np.cumsum(ns, out=goff[1:])
    m_in = np.rint(ns * deg_in / 2).astype(np.int64)
    m_out = np.where(bs > 1, np.rint(ns * deg_out / 2), 0).astype(np.int64)

    def per_draw(counts):
        gidx = np.repeat(np.arange(G, dtype=np.int64), counts)
        start = np.zeros(G + 1, dtype=np.int64)
        np.cumsum(counts, out=start[1:])
        local = np.arange(gidx.shape[0], dtype=np.int64) - start[gidx]
        return gidx, local

    def blocks_of(gidx, node):  # contiguous near-equal blocks: b(v) = floor(v * B / n) with a fix-up
        n_ = ns[gidx]
        B_ = bs[gidx]
        b = (node * B_) // n_
        # block_start(b) = floor(b * n / B); move to the block whose range holds node
        b = np.where((b + 1) * n_ // B_ <= node, b + 1, b)
        b = np.where(b * n_ // B_ > node, b - 1, b)
        return b, (b * n_) // B_, ((b + 1) * n_) // B_
    g1, i1 = per_draw(m_in)
    sd1 = sds[g1]
    u1 = (uniform01(sd1, 10, i1) * ns[g1]).astype(np.int64)
    b1, lo1, hi1 = blocks_of(g1, u1)
    v1 = lo1 + (uniform01(sd1, 11, i1) * (hi1 - lo1)).astype(np.int64)
    g2, i2 = per_draw(m_out)
    sd2 = sds[g2]
    u2 = (uniform01(sd2, 12, i2) * ns[g2]).astype(np.int64)
    b2, lo2, hi2 = blocks_of(g2, u2)
    bl2 = hi2 - lo2
    r = (uniform01(sd2, 13, i2) * (ns[g2] - bl2)).astype(np.int64)
    v2 = np.where(r >= lo2, r + bl2, r)
    # weights are drawn over each graph's concatenated (intra, inter) draw list
    wi1 = i1
    wi2 = m_in[g2] + i2
    w1 = uniform_int(sd1, 14, wi1, wmin, wmax)
    w2 = uniform_int(sd2, 14, wi2, wmin, wmax)
    gg_ = np.concatenate([g1, g2])
    u = np.concatenate([u1, u2]) + goff[gg_]
    v = np.concatenate([v1, v2]) + goff[gg_]
    w = np.concatenate([w1, w2])
    keep = u != v
    csr = from_edges(int(goff[-1]), u[keep], v[keep], w[keep])
    return goff.astype(np.int32), csr.row_ptr, csr.col, csr.w, sds


# ---------------------------------------------------------------------------
# Served workload: Poisson arrivals of R-MAT requests.
# ---------------------------------------------------------------------------
def served_stream(rate: float = 200.0, duration: float = 60.0, nmin: int = 1000,
                  nmax: int = 1000000, seed: int = 4):
    """List of (arrival_time_s, n, graph_seed): exponential inter-arrival times
    of mean 1/rate over ``duration`` seconds and node counts log-uniform in
    [nmin, nmax].  The graph of a request is ``rmat(scale=ceil(log2 n), n=n,
    draws=8n, wmax=8, seed=graph_seed)``."""
    out = []
    t = 0.0
    k = 0
    while True:
        r = float(uniform01(seed, 0, np.array([k]))[0])
        t += -math.log(1.0 - r) / rate
        if t >= duration:
            break
        r2 = float(uniform01(seed, 1, np.array([k]))[0])
        n = int(round(math.exp(math.log(nmin) + r2 * (math.log(nmax) - math.log(nmin)))))
        out.append((t, n, seed * 1000003 + k))
        k += 1
    return out


def served_graph(n: int, graph_seed: int) -> CSR:
    scale = max(1, int(math.ceil(math.log2(n))))
    return rmat(scale=scale, n=n, draws=8 * n, seed=graph_seed)


# ---------------------------------------------------------------------------
# Small structured and adversarial graphs.
# ---------------------------------------------------------------------------
def star(leaves: int, w: int = 1) -> CSR:
    u = np.zeros(leaves, dtype=np.int64)
    v = np.arange(1, leaves + 1, dtype=np.int64)
    return from_edges(leaves + 1, u, v, np.full(leaves, w))


def path(n: int) -> CSR:
    u = np.arange(n - 1, dtype=np.int64)
    return from_edges(n, u, u + 1)


def ring_of_cliques(r: int, k: int) -> CSR:
    """r cliques K_k; clique c's last node is joined to clique c+1's first node."""
    us, vs = [], []
    for c in range(r):
        base = c * k
        for i in range(k):
            for j in range(i + 1, k):
                us.append(base + i)
                vs.append(base + j)
        us.append(base + k - 1)
        vs.append(((c + 1) % r) * k)
    return from_edges(r * k, us, vs)


def two_cliques(k: int) -> CSR:
    """Two K_k joined by a single edge between node k-1 and node k."""
    us, vs = [], []
    for base in (0, k):
        for i in range(k):
            for j in range(i + 1, k):
                us.append(base + i)
                vs.append(base + j)
    us.append(k - 1)
    vs.append(k)
    return from_edges(2 * k, us, vs)


def random_small(n: int, p: float, seed: int, wmax: int = 4, loops: float = 0.0) -> CSR:
    """Erdos-Renyi-style graph with integer weights in [1, wmax] and optional
    self-loops (each node independently with probability ``loops``)."""
    iu, ju = np.triu_indices(n, 1)
    idx = iu.astype(np.int64) * n + ju
    keep = uniform01(seed, 0, idx) < p
    u, v = iu[keep].astype(np.int64), ju[keep].astype(np.int64)
    w = uniform_int(seed, 1, idx[keep], 1, wmax)
    if loops > 0:
        nodes = np.arange(n, dtype=np.int64)
        lk = uniform01(seed, 2, nodes) < loops
        u = np.concatenate([u, nodes[lk]])
        v = np.concatenate([v, nodes[lk]])
        w = np.concatenate([w, uniform_int(seed, 3, nodes[lk], 1, wmax)])
    return from_edges(n, u, v, w)


def isolated_and_loops(n: int, loops_every: int = 3) -> CSR:
    """n nodes, no edges between distinct nodes; every ``loops_every``-th node has a self-loop."""
    u = np.arange(0, n, loops_every, dtype=np.int64)
    return from_edges(n, u, u, np.full(u.shape[0], 2))


def directed_from_edges(n: int, u, v, w=None) -> CSR:
    """CSR of a directed graph: a draw (u, v, w) adds w to W_uv only (row u);
    duplicates are merged by summing.  Columns sorted, W need not be symmetric."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    w = np.ones(u.shape[0], np.int64) if w is None else np.asarray(w, dtype=np.int64)
    key = u * np.int64(max(n, 1)) + v
    order = np.argsort(key, kind="stable")
    key, w = key[order], w[order]
    if key.shape[0]:
        first = np.ones(key.shape[0], dtype=bool)
        first[1:] = key[1:] != key[:-1]
        starts = np.flatnonzero(first)
        ukey, uw = key[starts], np.add.reduceat(w, starts)
    else:
        ukey, uw = key, w
    rows = ukey // max(n, 1)
    counts = np.bincount(rows, minlength=n) if n else np.zeros(0, np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CSR(n, row_ptr.astype(np.int32), (ukey % max(n, 1)).astype(np.int32),
               uw.astype(np.int32))


def random_directed(n: int, p: float, seed: int, wmax: int = 4, loops: float = 0.0,
                    recip: float = 0.0) -> CSR:
    """Directed graph on n nodes: each ordered pair (i, j), i != j, is an arc
    with probability p; with probability `recip` an arc (i, j) also brings its
    reverse (j, i) with an independent weight; node i has a self-loop with
    probability `loops`.  Weights uniform in [1, wmax]."""
    i, j = np.meshgrid(np.arange(n, dtype=np.int64), np.arange(n, dtype=np.int64), indexing="ij")
    i, j = i.ravel(), j.ravel()
    pair = i * np.int64(max(n, 1)) + j
    arc = (uniform01(seed, 21, pair) < p) & (i != j)
    back = arc & (uniform01(seed, 22, pair) < recip)
    loop = (i == j) & (uniform01(seed, 23, pair) < loops)
    u = np.concatenate([i[arc], j[back], i[loop]])
    v = np.concatenate([j[arc], i[back], i[loop]])
    k = np.arange(u.shape[0], dtype=np.int64)
    return directed_from_edges(n, u, v, uniform_int(seed, 24, k, 1, wmax))


def cached(name: str, fn, *args, **kwargs):
    """Memoise a generator's CSR on disk under ``.graph_cache`` next to this package."""
    root = os.environ.get("SLM_GRAPH_CACHE") or os.path.join(
        os.path.dirname(os.path.dirname(os.path.abspath(__file__))), ".graph_cache")
    os.makedirs(root, exist_ok=True)
    path_ = os.path.join(root, name + ".npz")
    if os.path.exists(path_):
        z = np.load(path_)
        extra = z["extra"] if "extra" in z.files else None
        g = CSR(int(z["n"]), z["row_ptr"], z["col"], z["w"])
        return (g, extra) if extra is not None else g
    out = fn(*args, **kwargs)
    g, extra = (out if isinstance(out, tuple) else (out, None))
    tmp = path_ + ".tmp.npz"
    if extra is None:
        np.savez(tmp, n=g.n, row_ptr=g.row_ptr, col=g.col, w=g.w)
    else:
        np.savez(tmp, n=g.n, row_ptr=g.row_ptr, col=g.col, w=g.w, extra=extra)
    os.replace(tmp, path_)
    return out
