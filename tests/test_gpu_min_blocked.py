"""Hashmin's pull on the blocked edge layout (the layout of the blocked PageRank
pull, with the broadcast slots as codes and a shared-memory min per destination)
against the oracle, bit for bit with the per-superstep counts: forced, mixed with
the push modes superstep by superstep, on graphs with isolated vertices, hubs
and directed edges, and sharing one layout with PageRank on the same handle (the
bin tails switch between the two engines' neutral codes). The AUTO engine builds
the layout only after the handle's gather pulls have cost about as much."""
import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2010_08781_gb300 as ipg  # noqa: E402


def _check(G, ref, **opts):
    st = G.run("hashmin", **opts)
    got = G.values("hashmin")
    want, rst = ref
    assert st.halted and np.array_equal(got, want), int((got != want).sum())
    assert st.supersteps == rst["supersteps"]
    for k in ("active", "broadcasters", "messages"):
        assert getattr(st, k).tolist() == rst[k].tolist(), k
    return st


@pytest.fixture(scope="module")
def graphs():
    iso = inputs.rmat_graph(12, symmetrize=True, seed=4)
    s, t = iso.edges()
    return {
        "rmat14s": inputs.rmat_graph(14, symmetrize=True, seed=3),
        "rmat12d": inputs.rmat_graph(12, seed=5),  # directed: labels flow along out-edges
        "er": inputs.er_graph(20000, 60000, seed=6, symmetrize=True),
        "isolated": inputs.from_edges(iso.n + 5000, s, t),  # 5000 vertices without edges at the end
        "perm": inputs.rmat_graph(13, symmetrize=True, seed=7, permute_seed=9),
    }


@pytest.mark.parametrize("name", ["rmat14s", "rmat12d", "er", "isolated", "perm"])
@pytest.mark.parametrize("relabel", [False, True])
def test_blocked_min_pull_matches_oracle(graphs, name, relabel):
    g = graphs[name]
    ref = oracle.hashmin(g.n, g.row_ptr, g.col)
    with ipg.Graph.from_inputs(g, relabel=relabel) as G:
        _check(G, ref, policy="forced", forced_mode="pull", pr_engine="blocked")
        assert G.info()["bytes_blocked_layout"] > 0
        _check(G, ref, policy="forced", forced_mode="pull", pr_engine="blocked", use_graph=0)
        rng = np.random.default_rng(len(name))
        for _ in range(3):
            _check(G, ref, mode_sequence=rng.integers(0, 3, 9).tolist(), pr_engine="blocked")
        _check(G, ref, policy="threshold", pr_engine="blocked")
        _check(G, ref, policy="forced", forced_mode="pull", pr_engine="gather")  # the same handle, gather


def test_layout_shared_with_pagerank():
    """PageRank, Hashmin, PageRank again on one handle: each engine sets the bin
    tails it needs; both stay exact (PageRank within 1e-5)."""
    g = inputs.rmat_graph(13, symmetrize=True, seed=8)
    pr_want, _ = oracle.pagerank(g.n, g.row_ptr, g.col, T=30)
    hm_ref = oracle.hashmin(g.n, g.row_ptr, g.col)
    with ipg.Graph.from_inputs(g) as G:
        for _ in range(2):
            G.run("pagerank", policy="forced", forced_mode="pull", pr_engine="blocked")
            got = G.values("pagerank").astype(np.float64)
            assert float(np.max(np.abs(got - pr_want) / pr_want)) <= 1e-5
            _check(G, hm_ref, policy="forced", forced_mode="pull", pr_engine="blocked")


def test_auto_builds_the_layout_after_enough_gather_pulls():
    """AUTO on a graph of at least 2^26 edges: the first runs pull with the gather
    kernel; once the handle has run 6 gather pulls the next run builds the layout
    and uses it; the labels never change."""
    g = inputs.rmat_graph(22, symmetrize=True, seed=2)
    assert g.m >= 1 << 26
    ref = oracle.hashmin(g.n, g.row_ptr, g.col)
    with ipg.Graph.from_inputs(g) as G:
        pulls, built_at = 0, None
        for run in range(8):
            st = _check(G, ref, policy="forced", forced_mode="pull")
            if G.info()["bytes_blocked_layout"] and built_at is None:
                built_at = run
                assert pulls >= 6
            pulls += st.supersteps - 1
        assert built_at is not None and built_at <= 6 // (st.supersteps - 1) + 1
