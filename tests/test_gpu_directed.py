"""Directed graphs on the GPU (slm_create_graph_directed): the method on the
directed Q_w of Section 2.4 (out- and in-strengths), the setting of the
paper's experiments (Section 5.1, weighted directed LFR graphs).

Every whole run is compared level by level with the oracle's directed
restatement (oracle.directed_slm, pinned in tests/test_oracle_directed.py):
every level's ids and K, the per-level stats, every row of the sweep trace,
the final labels, and the final modularity with == (both sides divide the
same exact numerator once in FP64)."""
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


def _compose(r, l, n):
    lab = np.arange(n, dtype=np.int32)
    for t in range(l + 1):
        lab = r.levels[t][0][lab]
    return lab


def compare_directed(g, seed, P, max_sweeps=1000, flags=0):
    G = slm.Graph(g.row_ptr, g.col, g.w, directed=True)
    G.run(seed=seed, accept_p32=P, max_sweeps=max_sweeps, flags=flags)
    r = O.directed_slm(g, seed=seed, P=P, max_sweeps=max_sweeps, flags=flags)
    tr = G.trace()
    assert tr.shape == r.trace.shape and (tr == r.trace).all(), "per-sweep trace differs"
    assert G.num_levels() == r.num_levels
    for lv, (ids, K) in enumerate(r.levels):
        lab, k = G.partition(lv)
        assert k == K and np.array_equal(lab, ids), f"level {lv} differs"
        st = G.stats(lv)
        assert (st.sweeps, st.status, st.moves, st.splits, st.candidates,
                st.edges_scanned) == r.stats[lv], lv
        assert G.modularity(lv) == O.directed_modularity(g, _compose(r, lv, g.n))
    fin, _ = G.partition(-1)
    assert np.array_equal(fin, r.final)
    assert G.modularity(-1) == O.directed_modularity(g, r.final)
    G.close()
    return r


def small_digraphs():
    out = []
    for k in range(6):
        out.append((f"rand{k}", gg.random_directed(60 + 23 * k, 0.08, 300 + k, wmax=5,
                                                   loops=0.1 * (k % 3), recip=0.15 * (k % 4))))
    out.append(("sparse", gg.random_directed(400, 0.01, 7, wmax=3)))
    return out


DIGRAPHS = small_digraphs()


@pytest.mark.parametrize("name,g", DIGRAPHS, ids=[n for n, _ in DIGRAPHS])
@pytest.mark.parametrize("P", [O.P_HALF, O.P_ALWAYS], ids=["p_half", "p_one"])
def test_directed_full_run_small(name, g, P):
    compare_directed(g, seed=5, P=P)


def test_directed_no_positive_and_sweep_limit():
    g = gg.random_directed(300, 0.03, 17, wmax=4, loops=0.2)
    compare_directed(g, seed=2, P=O.P_HALF, flags=O.FLAG_NO_POSITIVE)
    compare_directed(g, seed=2, P=O.P_HALF, max_sweeps=2)


@pytest.mark.parametrize("mu_t,mu_w", [(0.2, 0.1), (0.5, 0.4)])
def test_directed_weighted_lfr_full_run(mu_t, mu_w):
    """The paper's benchmark family (directed weighted LFR-style, 10,000 nodes,
    mean degree 50) at two of its mixing pairs, complete runs."""
    g, _ = gg.lfr_directed(10000, mu_t, mu_w)
    compare_directed(g, seed=3, P=O.P_HALF)


def test_directed_weighted_lfr_high_mixing_bounded():
    """The third mixing pair (0.8, 0.7), where the method needs hundreds of
    sweeps: the first 30 sweeps of every level."""
    g, _ = gg.lfr_directed(10000, 0.8, 0.7)
    compare_directed(g, seed=3, P=O.P_HALF, max_sweeps=30)


def test_symmetric_graph_given_as_directed():
    """Every arc present both ways with equal weight: every directed value is
    twice the undirected one, so the decisions and partitions are the
    undirected run's."""
    g = gg.sbm_planted(n_blocks=6, block_size=80, p_in=0.15, p_out=0.01, seed=12)
    D = slm.Graph(g.row_ptr, g.col, g.w, directed=True)
    D.run(seed=4, accept_p32=slm.P_HALF)
    U = slm.Graph(g.row_ptr, g.col, g.w)
    U.run(seed=4, accept_p32=slm.P_HALF)
    assert D.num_levels() == U.num_levels()
    for lv in range(U.num_levels()):
        a, ka = D.partition(lv)
        b, kb = U.partition(lv)
        assert ka == kb and np.array_equal(a, b)
    assert (D.trace() == U.trace()).all()
    assert abs(D.modularity(-1) - U.modularity(-1)) < 1e-12


def test_directed_invalid_inputs():
    def make(rp, col, w=None):
        return slm.Graph(np.array(rp, np.int32), np.array(col, np.int32),
                         None if w is None else np.array(w, np.int32), directed=True)
    with pytest.raises(slm.SlmError) as e:
        make([0, 2, 2], [1, 1])                      # duplicated column
    assert e.value.name == "SLM_ERR_INVALID_ARGUMENT"
    with pytest.raises(slm.SlmError) as e:
        make([0, 1, 1], [1], [0])                    # weight <= 0
    assert e.value.name == "SLM_ERR_INVALID_ARGUMENT"
    with pytest.raises(slm.SlmError) as e:
        make([0, 1, 1], [2])                         # column out of range
    assert e.value.name == "SLM_ERR_INVALID_ARGUMENT"
    with pytest.raises(slm.SlmError) as e:
        make([0, 1, 2], [1, 0], [1 << 29, 1 << 29])  # m_w = 2^30
    assert e.value.name == "SLM_ERR_OVERFLOW"
    G = make([0, 1, 1], [1], [3])                    # one arc: no positive gain, as the oracle finds
    G.run(seed=1, accept_p32=slm.P_HALF)
    lab, K = G.partition(-1)
    r = O.directed_slm(gg.directed_from_edges(2, [0], [1], [3]), seed=1, P=O.P_HALF)
    assert np.array_equal(lab, r.final)
    assert slm.load().slm_graph_is_directed(G._h) == 1
    G.close()
