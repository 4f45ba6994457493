"""Unit-weight SSSP (Fig. 10 exactly: every edge weighs 1, i.e. BFS levels) on the
GPU against the oracle, bit for bit with the per-superstep counts: pull with the
direction-optimising early exit (the first in-neighbour that broadcast in the
last superstep decides the vertex) and without it, both push modes, random mode
sequences, the degree bins at their extremes, and R-MAT graphs whose vertex ids
were randomly permuted (hubs spread over the id range), with and without the
library's degree-class renumbering."""
import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2010_08781_gb300 as ipg  # noqa: E402


def _check(G, g, ref, **opts):
    st = G.run("sssp", **opts)
    got = G.values("sssp")
    want, rst = ref
    assert st.halted and np.array_equal(got, want), int((got != want).sum())
    assert st.supersteps == rst["supersteps"]
    for k in ("active", "broadcasters", "messages"):
        assert getattr(st, k).tolist() == rst[k].tolist(), k
    return st


@pytest.fixture(scope="module")
def unit_graphs():
    return {
        "rmat13s": inputs.rmat_graph(13, symmetrize=True, seed=5),
        "rmat13s_perm": inputs.rmat_graph(13, symmetrize=True, seed=5, permute_seed=11),
        "rmat12d_perm": inputs.rmat_graph(12, seed=6, permute_seed=3),
        "er": inputs.er_graph(5000, 20000, seed=8),
    }


@pytest.mark.parametrize("name", ["rmat13s", "rmat13s_perm", "rmat12d_perm", "er"])
@pytest.mark.parametrize("relabel", [False, True])
def test_unit_weight_sssp_every_mode(unit_graphs, name, relabel):
    g = unit_graphs[name]
    assert g.w is None
    src = int(np.argmax(g.out_degree()))  # a hub: a deep frontier in few supersteps
    ref = oracle.sssp(g.n, g.row_ptr, g.col, None, source=src)
    with ipg.Graph.from_inputs(g, relabel=relabel) as G:
        for mode in ("pull", "push_dense", "push_sparse"):
            _check(G, g, ref, source=src, policy="forced", forced_mode=mode)
        _check(G, g, ref, source=src, policy="forced", forced_mode="pull", pull_early_exit=0)
        _check(G, g, ref, source=src, policy="forced", forced_mode="pull", use_graph=0)
        for t1, t2 in ((1, 2), (64, 100000)):  # every vertex in the CTA bin / in lane tiles
            _check(G, g, ref, source=src, policy="forced", forced_mode="pull", t1=t1, t2=t2)
        rng = np.random.default_rng(len(name))
        _check(G, g, ref, source=src, mode_sequence=rng.integers(0, 3, 11).tolist())
        _check(G, g, ref, source=src, policy="threshold")


def test_unit_weight_bfs_layers_and_unreachable():
    """Distances are the BFS layers; vertices of another component stay INF."""
    a = inputs.path(50)
    b = inputs.rmat_graph(8, symmetrize=True, seed=2)
    s = np.concatenate([a.edges()[0], b.edges()[0] + 50])
    t = np.concatenate([a.edges()[1], b.edges()[1] + 50])
    g = inputs.from_edges(50 + b.n, s, t)
    ref = oracle.sssp(g.n, g.row_ptr, g.col, None, source=0)
    assert ref[0][:50].tolist() == list(range(50)) and (ref[0][50:] == ipg.INF).all()
    with ipg.Graph.from_inputs(g) as G:
        for mode in ("pull", "push_sparse"):
            _check(G, g, ref, source=0, policy="forced", forced_mode=mode)
