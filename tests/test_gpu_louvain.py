"""Colour-synchronous Louvain on the GPU (slm_run_louvain), the comparison
method of Section 6, against the oracle's restatement (oracle.louvain_colour,
pinned in tests/test_oracle_louvain_colour.py).

Every run is compared level by level: each level's ids and K, the per-level
stats, every row of the pass trace, the final labels, and the final
modularity with == (both sides divide the same exact numerator once)."""
import numpy as np
import pytest

import graphgen as gg
import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1702_04645_gb300 as slm  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def lib():
    slm.build()
    return slm.load()


def compare_louvain(g, seed=1, max_passes=1000, max_levels=64):
    G = slm.Graph(g.row_ptr, g.col, g.w)
    G.run_louvain(seed=seed, max_passes=max_passes, max_levels=max_levels)
    r = O.louvain_colour(g, seed=seed, max_passes=max_passes, max_levels=max_levels)
    tr = G.trace()
    assert tr.shape == r.trace.shape and (tr == r.trace).all(), "pass trace differs"
    assert G.num_levels() == r.num_levels
    for lv, (ids, K) in enumerate(r.levels):
        lab, k = G.partition(lv)
        assert k == K and np.array_equal(lab, ids), f"level {lv} differs"
        st = G.stats(lv)
        assert (st.sweeps, st.status, st.moves, st.splits, st.candidates,
                st.edges_scanned) == r.stats[lv], lv
    fin, _ = G.partition(-1)
    assert np.array_equal(fin, r.final)
    assert G.modularity(-1) == O.modularity(g, r.final)
    G.close()
    return r


def small_graphs():
    out = [(f"rand{s}", gg.random_small(40 + 17 * s, 0.1, 400 + s, wmax=5,
                                        loops=0.2 if s % 2 else 0.0)) for s in range(5)]
    out.append(("ties", gg.random_small(120, 0.05, 77, wmax=1)))
    out.append(("sbm", gg.sbm_planted(n_blocks=8, block_size=60, p_in=0.2, p_out=0.01, seed=9)))
    out.append(("ring", gg.ring_of_cliques(40, 5)))
    out.append(("star", gg.star(300)))
    out.append(("loops", gg.isolated_and_loops(50)))
    return out


GRAPHS = small_graphs()


@pytest.mark.parametrize("name,g", GRAPHS, ids=[n for n, _ in GRAPHS])
@pytest.mark.parametrize("seed", [1, 6])
def test_louvain_small_graphs(name, g, seed):
    compare_louvain(g, seed=seed)


@pytest.mark.parametrize("mu_t,mu_w", [(0.2, 0.1), (0.5, 0.4), (0.8, 0.7)])
def test_louvain_weighted_lfr(mu_t, mu_w):
    """The paper's benchmark family (weighted LFR-style, 10,000 nodes, mean
    degree 50), symmetric form, at its three mixing pairs."""
    g, _ = gg.lfr_weighted(10000, mu_t, mu_w)
    compare_louvain(g, seed=3)


def test_louvain_rmat_hubs():
    """R-MAT scale 14: hub rows take the scan's hub path inside one colour
    class."""
    g = gg.rmat(14, seed=5)
    compare_louvain(g, seed=2)


def test_louvain_rmat_layout_path():
    """R-MAT scale 17 (131,072 nodes): the large colour classes of level 0
    (more than 8,192 nodes) and the classes holding hub rows run the MAXIMAL
    scan on their own bucketed layouts, the others take the direct decision,
    one block per node."""
    g = gg.rmat(17, seed=2)
    compare_louvain(g, seed=4)


def test_louvain_rmat_threshold_stops():
    """R-MAT scale 16: the levels end on the numerator threshold (status 1)
    after passes whose moves undo one another."""
    g = gg.rmat(16, seed=2)
    r = compare_louvain(g, seed=1)
    assert any(st[1] == 1 for st in r.stats)


def test_louvain_limits_and_results():
    g = gg.sbm_planted(n_blocks=6, block_size=50, p_in=0.25, p_out=0.02, seed=4)
    r = compare_louvain(g, max_passes=1)
    assert r.stats[0][0] == 1 and r.stats[0][1] == 2
    compare_louvain(g, max_levels=1)
    compare_louvain(g, max_levels=0)
    # the method's run and the comparison run replace each other's results
    G = slm.Graph(g.row_ptr, g.col, g.w)
    G.run(seed=1, accept_p32=slm.P_HALF)
    a = G.partition(-1)[0].copy()
    G.run_louvain(seed=1)
    assert np.array_equal(G.partition(-1)[0], O.louvain_colour(g, seed=1).final)
    G.run(seed=1, accept_p32=slm.P_HALF)
    assert np.array_equal(G.partition(-1)[0], a)
    G.close()


def test_louvain_invalid_inputs():
    g = gg.sbm_planted(n_blocks=3, block_size=20, p_in=0.3, p_out=0.05, seed=1)
    G = slm.Graph(g.row_ptr, g.col, g.w)
    G.run_louvain(seed=1)
    before = G.partition(-1)[0].copy()
    for kw in (dict(max_passes=0), dict(max_passes=70000), dict(max_levels=-1)):
        with pytest.raises(slm.SlmError) as e:
            G.run_louvain(seed=1, **kw)
        assert e.value.name == "SLM_ERR_INVALID_ARGUMENT"
        assert np.array_equal(G.partition(-1)[0], before)  # previous results kept
    G.close()
    D = slm.Graph(g.row_ptr, g.col, g.w, directed=True)
    with pytest.raises(slm.SlmError) as e:
        D.run_louvain(seed=1)
    assert e.value.name == "SLM_ERR_INVALID_ARGUMENT"
    D.close()


@pytest.mark.parametrize("n", [0, 1, 7])
def test_louvain_degenerate(n):
    g = gg.from_edges(n, [], [])
    G = slm.Graph(g.row_ptr, g.col, g.w)
    G.run_louvain(seed=1)
    assert G.num_levels() == 0
    assert np.array_equal(G.partition(-1)[0], np.arange(n))
    G.close()
