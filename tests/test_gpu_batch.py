"""The batched form: every graph of a forest gives, bit for bit, what the oracle
(and the single-graph path) gives for that graph alone with its seed."""
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


def mixed_graphs():
    gs = [gg.two_cliques(5), gg.ring_of_cliques(12, 4), gg.path(120), gg.star(400),
          gg.isolated_and_loops(9), gg.from_edges(1, [], []), gg.random_small(60, 0.1, 3, wmax=5, loops=0.2)]
    for n, b, sd in gg.forest_sbm_params(num_graphs=10, nmin=100, nmax=3000, seed_base=1000):
        gs.append(gg.forest_sbm_graph(n, b, sd))
    gs.append(gg.rmat(scale=10, seed=11))
    return gs


def check_graph_against_oracle(B, k, g, seed, P, **kw):
    r = O.slm(g, seed=seed, P=P, **kw)
    assert B.num_levels(k) == r.num_levels, k
    for l, (ids, K) in enumerate(r.levels):
        lab, kk = B.partition(k, l)
        assert kk == K and (lab == ids).all(), (k, l)
        st = B.stats(k, l)
        assert (st.sweeps, st.status, st.moves, st.splits, st.candidates, st.edges_scanned) == r.stats[l], (k, l)
    fin, _ = B.partition(k, -1)
    assert (fin == r.final).all(), k
    assert B.modularity(k) == O.modularity(g, r.final), k


@pytest.mark.parametrize("P", [O.P_HALF, O.P_ALWAYS], ids=["p_half", "p_one"])
def test_forest_equals_each_graph_alone(P):
    gs = mixed_graphs()
    seeds = np.arange(len(gs), dtype=np.uint64) * 7 + 3
    B = slm.Batch(gs, seeds=seeds).run(accept_p32=P)
    for k, g in enumerate(gs):
        check_graph_against_oracle(B, k, g, int(seeds[k]), P)
        G = slm.Graph(g.row_ptr, g.col, g.w).run(seed=int(seeds[k]), accept_p32=P)
        fin, _ = G.partition(-1)
        assert (fin == B.partition(k, -1)[0]).all()


def test_forest_result_does_not_depend_on_company():
    gs = mixed_graphs()
    seeds = np.arange(len(gs), dtype=np.uint64) + 100
    full = slm.Batch(gs, seeds=seeds).run()
    order = [5, 2, 17, 0, 9]
    sub = slm.Batch([gs[k] for k in order], seeds=seeds[order]).run()
    for j, k in enumerate(order):
        assert (sub.partition(j, -1)[0] == full.partition(k, -1)[0]).all()
        assert sub.modularity(j) == full.modularity(k)


def test_forest_sweep_and_level_limits():
    gs = mixed_graphs()[:8]
    B = slm.Batch(gs).run(seed=4, max_sweeps=2, max_levels=1)
    for k, g in enumerate(gs):
        check_graph_against_oracle(B, k, g, 4, O.P_HALF, max_sweeps=2, max_levels=1)


def test_forest_rejects_edges_across_graphs():
    a, b = gg.random_small(10, 0.4, 1), gg.random_small(12, 0.4, 2)
    goff, rp, col, w = slm.pack_forest([a, b])
    col = col.copy()
    col[0] = 15  # row 0 of graph 0 now points into graph 1 (and loses symmetry)
    with pytest.raises(slm.SlmError):
        slm.Batch(graph_off=goff, row_ptr=rp, col=col, w=w)
