"""The benchmark-sized graphs on the GPU: R-MAT scale 20 (1,048,576 nodes) and
the LFR-style graph (4,194,304 nodes).

At these sizes the oracle cannot redo a whole run inside the test suite's
time, so the checks are
  * sampled outputs recomputed one node at a time from the definitions
    (ASSIGN's best neighbour, the MAXIMAL scan's best community, gain and
    local gain), on the same launch configuration slm_run uses;
  * properties that hold at any size: the final modularity equals the oracle's
    modularity of the GPU's own final partition (exact integer numerator, one
    FP64 division), every level's labels are 0..K-1, the last level stopped
    for a stated reason, and strengths and m_w are preserved;
  * with SLM_FULL_ORACLE=1 in the environment, the complete oracle run,
    compared level by level (minutes of single-threaded CPU time).
"""
import os

import numpy as np
import pytest

import graphgen as gg
import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1702_04645_gb300 as slm  # noqa: E402

SAMPLES = 1500


@pytest.fixture(scope="module", autouse=True)
def lib():
    slm.build()
    return slm.load()


def _rmat():
    return gg.cached("rmat_s20_seed2", gg.rmat, scale=20, seed=2)


def _lfr():
    return gg.cached("lfr_style_default", lambda: gg.lfr_style()[0])


GRAPHS = {"rmat_s20": _rmat, "lfr_4m": _lfr}


@pytest.fixture(scope="module", params=list(GRAPHS))
def big(request):
    g = GRAPHS[request.param]()
    return request.param, g


def _sample(g, seed):
    rng = np.random.default_rng(seed)
    deg = np.diff(g.row_ptr)
    nz = np.nonzero(deg)[0]
    pick = rng.choice(nz, size=min(SAMPLES, nz.shape[0]), replace=False)
    # always include the largest rows (the hub shape)
    hubs = np.argsort(deg)[-20:]
    return np.unique(np.concatenate([pick, hubs]))


def _strengths(g):
    row = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    return np.bincount(row, weights=g.w, minlength=g.n).astype(np.int64)  # exact: m_w < 2^31


def test_assign_sampled(big):
    name, g = big
    rp, col, w = (torch.from_numpy(x).cuda() for x in (g.row_ptr, g.col, g.w))
    s_d, m = slm.step_strengths(rp, col, w)
    a = slm.step_assign(rp, col, w, s_d, m).cpu().numpy()
    s = _strengths(g)
    assert int(s.sum()) == m
    for i in _sample(g, 1):
        lo, hi = g.row_ptr[i], g.row_ptr[i + 1]
        j = g.col[lo:hi].astype(np.int64)
        wv = g.w[lo:hi].astype(np.int64)
        keep = j != i
        j, wv = j[keep], wv[keep]
        if j.shape[0] == 0:
            assert a[i] == i
            continue
        sc = m * wv - s[i] * s[j]
        best = sc.max()
        exp = int(j[sc == best].min()) if best > 0 else int(i)
        assert a[i] == exp, (name, int(i))


def test_scan_sampled(big):
    name, g = big
    rp, col, w = (torch.from_numpy(x).cuda() for x in (g.row_ptr, g.col, g.w))
    s_d, m = slm.step_strengths(rp, col, w)
    a = slm.step_assign(rp, col, w, s_d, m)
    a, root_d, _ = slm.step_positive(rp, col, w, s_d, m, a)
    best, gain, gl = (t.cpu().numpy() for t in slm.step_scan(rp, col, w, s_d, m, root_d))
    root = root_d.cpu().numpy().astype(np.int64)
    s = _strengths(g)
    sigma = np.bincount(root, weights=s, minlength=g.n).astype(np.int64)
    for i in _sample(g, 2):
        lo, hi = g.row_ptr[i], g.row_ptr[i + 1]
        j = g.col[lo:hi].astype(np.int64)
        wv = g.w[lo:hi].astype(np.int64)
        keep = j != i
        cs, inv = np.unique(root[j[keep]], return_inverse=True)
        kic = np.bincount(inv, weights=wv[keep], minlength=cs.shape[0]).astype(np.int64)
        ci = root[i]
        own = int(kic[cs == ci].sum())
        g_own = m * own - int(s[i]) * (int(sigma[ci]) - int(s[i]))
        other = cs != ci
        exp_best, exp_gain = ci, 0
        if other.any():
            sc = m * kic[other] - int(s[i]) * sigma[cs[other]]
            top = sc.max()
            c_top = int(cs[other][sc == top].min())
            if top - g_own > 0:
                exp_best, exp_gain = c_top, int(top - g_own)
        assert gl[i] == g_own, (name, int(i))
        assert best[i] == exp_best and gain[i] == exp_gain, (name, int(i))


@pytest.fixture(scope="module")
def runs():
    # a whole run at full size is checked on the R-MAT graph; on the LFR-style
    # graph the method needs many minutes (POSITIVE peels its large
    # communities one branch at a time), beyond a test suite's budget
    g = _rmat()
    G = slm.Graph(g.row_ptr, g.col, g.w)
    G.run(seed=1, accept_p32=slm.P_HALF)
    return "rmat_s20", g, G


def test_run_properties(runs):
    name, g, G = runs
    lab, K = G.partition(-1)
    assert lab.shape[0] == g.n and lab.min() >= 0 and lab.max() == K - 1
    assert np.unique(lab).shape[0] == K
    assert G.modularity(-1) == O.modularity(g, lab)
    for lv in range(G.num_levels()):
        ids, Kl = G.partition(lv)
        st = G.stats(lv)
        assert ids.shape[0] == st.n and np.unique(ids).shape[0] == Kl == st.n_communities
        assert st.status in (0, 1, 2)
    top = G.stats(-1)
    assert top.status in (0, 1) and top.n_communities == top.n


def test_lfr_bounded_run():
    """The LFR-style graph with at most 5 sweeps per level and 3 levels (the
    method does not settle on it: the oracle on a 16,384-node graph of the same
    recipe reaches the 1,000-sweep limit at level 0): the run stops at the
    limits with consistent levels and the oracle's modularity of the GPU
    partition."""
    g = _lfr()
    G = slm.Graph(g.row_ptr, g.col, g.w)
    G.run(seed=1, accept_p32=slm.P_HALF, max_sweeps=5, max_levels=3)
    lab, K = G.partition(-1)
    assert lab.shape[0] == g.n and np.unique(lab).shape[0] == K
    assert G.modularity(-1) == O.modularity(g, lab)
    for lv in range(G.num_levels()):
        st = G.stats(lv)
        assert st.sweeps <= 5 and st.status in (0, 1, 2)
    G.close()


@pytest.mark.skipif(os.environ.get("SLM_FULL_ORACLE") != "1",
                    reason="complete oracle run at full size: set SLM_FULL_ORACLE=1")
def test_full_oracle(runs):
    name, g, G = runs
    r = O.slm(g, seed=1, P=O.P_HALF)
    assert G.num_levels() == r.num_levels
    for lv, (ids, K) in enumerate(r.levels):
        lab, k = G.partition(lv)
        assert k == K and np.array_equal(lab, ids), (name, lv)
    fin, _ = G.partition(-1)
    assert np.array_equal(fin, r.final)
    assert G.modularity(-1) == O.modularity(g, r.final)
