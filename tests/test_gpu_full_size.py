"""The benchmark-sized graphs on the GPU: R-MAT scale 20 (1,048,576 nodes) and
the LFR-style graph (4,194,304 nodes), plus a 262,144-node graph of the
LFR-style recipe.

  * ASSIGN's best neighbour and the MAXIMAL scan's best community, gain and
    local gain of EVERY node are recomputed from the definitions with
    vectorised numpy (exact int64) and compared element by element, on the
    launch configuration slm_run uses;
  * whole runs are compared level by level (every level's ids, K, stats, the
    per-sweep trace, the final labels and Q) with the oracle's runs stored
    under tests/golden/ by tests/golden/make_run_goldens.py (which calls
    only the oracle): the complete run on the R-MAT graph, and bounded runs
    (3 sweeps per level at 262,144 nodes; 2 sweeps per level, for level 0
    alone and for three levels, at 4,194,304) on the LFR-style graphs, where the method does not settle:
    after a few sweeps long assignment cycles form, whose cycle cuts cost
    the oracle hours;
  * properties that hold at any size: every level's labels are 0..K-1, the
    last level stopped for a stated reason, and the final modularity equals
    the oracle's modularity of the GPU's own final partition.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle as O
from whole_array import expected_assign, expected_scan, strengths as _strengths

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1702_04645_gb300 as slm  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def lib():
    slm.build()
    return slm.load()


def _rmat():
    return gg.cached("rmat_s20_seed2", gg.rmat, scale=20, seed=2)


def _lfr():
    return gg.cached("lfr_style_default", lambda: gg.lfr_style()[0])


def _lfr_256k():
    return gg.cached("lfr_style_n262144", lambda: gg.lfr_style(n=262144)[0])


GRAPHS = {"rmat_s20": _rmat, "lfr_4m": _lfr}


@pytest.fixture(scope="module", params=list(GRAPHS))
def big(request):
    g = GRAPHS[request.param]()
    return request.param, g


def _sha(x) -> str:
    return hashlib.sha256(np.ascontiguousarray(x, dtype="<i4").tobytes()).hexdigest()


def test_assign_all_nodes(big):
    name, g = big
    rp, col, w = (torch.from_numpy(x).cuda() for x in (g.row_ptr, g.col, g.w))
    s_d, m = slm.step_strengths(rp, col, w)
    a = slm.step_assign(rp, col, w, s_d, m).cpu().numpy()
    exp, s, m_host = expected_assign(g)
    assert m == m_host
    assert np.array_equal(s_d.cpu().numpy().astype(np.int64), s)
    bad = np.nonzero(a != exp)[0]
    assert bad.shape[0] == 0, (name, bad[:10])


def test_scan_all_nodes(big):
    name, g = big
    rp, col, w = (torch.from_numpy(x).cuda() for x in (g.row_ptr, g.col, g.w))
    s_d, m = slm.step_strengths(rp, col, w)
    a = slm.step_assign(rp, col, w, s_d, m)
    a, root_d, _ = slm.step_positive(rp, col, w, s_d, m, a)
    best, gain, gl = (t.cpu().numpy() for t in slm.step_scan(rp, col, w, s_d, m, root_d))
    s = _strengths(g)
    eb, eg, el = expected_scan(g, root_d.cpu().numpy(), s, m)
    for what, got, exp in (("local gain", gl, el), ("best", best, eb), ("gain", gain, eg)):
        bad = np.nonzero(got.astype(np.int64) != exp)[0]
        assert bad.shape[0] == 0, (name, what, bad[:10])


def _golden(case):
    with open(os.path.join(GOLDEN, f"run_{case}.json")) as f:
        return json.load(f)


def compare_with_golden(g, gold, **run_kw):
    fp = gold["graph"]
    assert (g.n, g.nnz) == (fp["n"], fp["nnz"]), "the generator no longer makes the stored graph"
    assert _sha(g.row_ptr) == fp["row_ptr"] and _sha(g.col) == fp["col"] and _sha(g.w) == fp["w"]
    opts = gold["options"]
    G = slm.Graph(g.row_ptr, g.col, g.w, directed=gold.get("method") == "directed_slm")
    if gold.get("method", "slm") == "louvain_colour":
        G.run_louvain(seed=opts["seed"], max_passes=opts.get("max_passes", 1000),
                      max_levels=opts.get("max_levels", 64), **run_kw)
    else:
        G.run(seed=opts["seed"], accept_p32=opts["P"], max_sweeps=opts.get("max_sweeps", 1000),
              max_levels=opts.get("max_levels", 64), **run_kw)
    tr = G.trace()
    exp_tr = np.array(gold["trace"], dtype=np.int64).reshape(-1, 6)
    assert tr.shape == exp_tr.shape, ("sweeps", tr.shape, exp_tr.shape)
    rows = np.nonzero((tr != exp_tr).any(axis=1))[0]
    assert rows.shape[0] == 0, ("first differing sweep", tr[rows[0]].tolist(), exp_tr[rows[0]].tolist())
    assert G.num_levels() == len(gold["levels"])
    for lv, exp in enumerate(gold["levels"]):
        ids, K = G.partition(lv)
        st = G.stats(lv)
        assert (st.n, K) == (exp["n"], exp["K"]), lv
        assert _sha(ids) == exp["ids"], f"level {lv} ids differ"
        assert [st.sweeps, st.status, st.moves, st.splits, st.candidates,
                st.edges_scanned] == exp["stats"], lv
    fin, K = G.partition(-1)
    assert _sha(fin) == gold["final"]["labels"] and K == gold["final"]["K"]
    q = G.modularity(-1)
    assert q == float.fromhex(gold["q"])           # same exact numerator, one FP64 division
    return G


def test_rmat_s20_whole_run_equals_oracle():
    """The benchmark run (R-MAT scale 20, seed 1, p = 1/2, no limits) equals
    the oracle's complete run level by level, with every sweep of the trace:
    this covers ASSIGN, POSITIVE (incremental rounds), branch gains, targets,
    the touched-set COMPONENTS and POSITIVE passes and AGGREGATE at the size
    where their thresholds switch."""
    G = compare_with_golden(_rmat(), _golden("rmat_s20"))
    G.close()


def test_directed_lfr_high_mixing_whole_run_equals_oracle():
    """The directed weighted LFR-style graph of 10,000 nodes at the paper's
    highest mixing pair (0.8, 0.7), a whole run with the default limits: level
    0 stops at the 1,000-sweep limit (long assignment cycles, tens of
    thousands of POSITIVE rounds), then two more levels; every sweep equals
    the directed oracle's, stored after 697 s of oracle time."""
    g, _ = gg.lfr_directed(10000, 0.8, 0.7)
    G = compare_with_golden(g, _golden("lfr_directed_1e4_high_mixing"))
    G.close()


def test_louvain_rmat_s20_whole_run_equals_oracle():
    """The comparison method (colour-synchronous Louvain, colouring seed 1)
    on the benchmark graph equals the oracle's complete run: every level's
    colouring-driven passes, the threshold stops and AGGREGATE."""
    G = compare_with_golden(_rmat(), _golden("louvain_rmat_s20"))
    G.close()


def test_rmat_s20_whole_run_timed_flags_equal():
    """The timed run the benchmark makes (phase timers on) gives the same result."""
    G = compare_with_golden(_rmat(), _golden("rmat_s20"), flags=slm.FLAG_TIMING)
    G.close()


def test_lfr_4m_three_levels_run_equals_oracle():
    """The 4,194,304-node LFR-style graph through three levels with at most 2
    sweeps each (ASSIGN, COMPONENTS, POSITIVE and two corrections per level,
    then AGGREGATE of each level graph) equals the oracle's run, stored
    after 6,991 s of oracle time."""
    G = compare_with_golden(_lfr(), _golden("lfr_4m_bounded"))
    G.close()


def test_lfr_4m_level0_run_equals_oracle():
    """The 4,194,304-node LFR-style graph, level 0 with at most 2 sweeps
    (ASSIGN, COMPONENTS, the first POSITIVE over the whole graph, two MAXIMAL
    corrections with their POSITIVE calls), equals the oracle's run: the
    level's ids, stats, both sweeps of the trace and Q.  Deeper runs form
    long assignment cycles whose cuts take the oracle hours at this size."""
    G = compare_with_golden(_lfr(), _golden("lfr_4m_level0"))
    G.close()


def test_lfr_256k_bounded_run_equals_oracle():
    """A 262,144-node graph of the LFR-style recipe with at most 3 sweeps per
    level, every level, equals the oracle's run."""
    G = compare_with_golden(_lfr_256k(), _golden("lfr_256k_bounded"))
    G.close()


def test_run_properties():
    g = _rmat()
    G = slm.Graph(g.row_ptr, g.col, g.w)
    G.run(seed=1, accept_p32=slm.P_HALF)
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
    G.close()
