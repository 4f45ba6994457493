"""SSSP's pull on the blocked edge layout against the oracle, bit for bit with
the per-superstep counts. SSSP's message adds the edge weight to the broadcast
distance (Fig. 10 with weights), so the layout keeps each entry's weight beside
its source (one byte: graphs whose weights are below 256) and the scatter writes
distance + weight as the entry's code; on unweighted graphs it adds 1. Graphs with
a weight of 256 or more keep the gather pull, whatever the engine option asks,
and build no layout for it. Covered: weighted and unweighted, directed and
symmetric, renumbered or not, several sources (a hub, a leaf, an isolated vertex),
forced pull and random mode sequences, a layout first built by PageRank or by
Hashmin on the same handle, and the AUTO engine after the handle's gather pulls."""
import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2010_08781_gb300 as ipg  # noqa: E402


def _check(G, ref, source, **opts):
    st = G.run("sssp", source=source, **opts)
    got = G.values("sssp")
    want, rst = ref
    assert st.halted and np.array_equal(got, want), int((got != want).sum())
    assert st.supersteps == rst["supersteps"]
    for k in ("active", "broadcasters", "messages"):
        assert getattr(st, k).tolist() == rst[k].tolist(), k
    return st


def _ref(g, source):
    return oracle.sssp(g.n, g.row_ptr, g.col, g.w, source=source)


@pytest.fixture(scope="module")
def graphs():
    iso = inputs.rmat_graph(12, symmetrize=True, weighted=True, seed=4)
    s, t = iso.edges()
    out = {
        "rmat14sw": inputs.rmat_graph(14, symmetrize=True, weighted=True, seed=3),
        "rmat13s": inputs.rmat_graph(13, symmetrize=True, seed=5),          # unweighted: + 1
        "rmat12dw": inputs.rmat_graph(12, weighted=True, seed=6),           # directed
        "isolated": inputs.from_edges(iso.n + 3000, s, t, weighted=True),   # 3000 vertices without edges
        "perm": inputs.rmat_graph(13, symmetrize=True, weighted=True, seed=7, permute_seed=9),
    }
    return out


@pytest.mark.parametrize("name", ["rmat14sw", "rmat13s", "rmat12dw", "isolated", "perm"])
@pytest.mark.parametrize("relabel", [False, True])
def test_blocked_sssp_matches_oracle(graphs, name, relabel):
    g = graphs[name]
    if g.w is not None:
        assert int(g.w.max()) <= 255
    deg = np.diff(g.row_ptr)
    sources = [int(np.argmax(deg)), int(np.argmin(deg[: g.n // 2] + (deg[: g.n // 2] == 0) * 10**9)), g.n - 1]
    with ipg.Graph.from_inputs(g, relabel=relabel) as G:
        for i, src in enumerate(sources):
            ref = _ref(g, src)
            _check(G, ref, src, policy="forced", forced_mode="pull", pr_engine="blocked")
            assert G.info()["bytes_blocked_layout"] > 0
            rng = np.random.default_rng(i + len(name))
            for _ in range(2):
                _check(G, ref, src, mode_sequence=rng.integers(0, 3, 9).tolist(), pr_engine="blocked")
            _check(G, ref, src, policy="threshold", pr_engine="blocked")
            _check(G, ref, src, policy="forced", forced_mode="pull", pr_engine="gather")


def test_layout_built_by_pagerank_or_hashmin_serves_sssp():
    g = inputs.rmat_graph(13, symmetrize=True, weighted=True, seed=8)
    ref = _ref(g, 0)
    hm = oracle.hashmin(g.n, g.row_ptr, g.col)[0]
    pr, _ = oracle.pagerank(g.n, g.row_ptr, g.col, T=30)
    for first in ("pagerank", "hashmin"):
        with ipg.Graph.from_inputs(g) as G:
            G.run(first, policy="forced", forced_mode="pull", pr_engine="blocked")
            b = G.info()["bytes_blocked_layout"]
            assert b > 0
            _check(G, ref, 0, policy="forced", forced_mode="pull", pr_engine="blocked")
            assert G.info()["bytes_blocked_layout"] == b  # the same layout
            G.run("hashmin", policy="forced", forced_mode="pull", pr_engine="blocked")
            assert np.array_equal(G.values("hashmin"), hm)
            G.run("pagerank", policy="forced", forced_mode="pull", pr_engine="blocked")
            got = G.values("pagerank").astype(np.float64)
            assert float(np.max(np.abs(got - pr) / pr)) <= 1e-5
            _check(G, ref, 0, policy="forced", forced_mode="pull", pr_engine="blocked")


def test_heavy_weights_keep_the_gather_pull():
    """A weight of 256 or more: no byte per entry holds it, so the pull gathers (the
    values stay exact) and no layout is built for SSSP; a layout built by another
    program holds no weights and is not used by SSSP either."""
    g = inputs.rmat_graph(12, symmetrize=True, weighted=True, seed=9)
    w = g.w.copy()
    i = len(w) // 2  # edge (u, v) and its reverse (v, u) both weigh 300
    u = int(np.searchsorted(g.row_ptr, i, side="right") - 1)
    v = int(g.col[i])
    j = int(g.row_ptr[v]) + int(np.nonzero(g.col[g.row_ptr[v]:g.row_ptr[v + 1]] == u)[0][0])
    w[i] = w[j] = 300
    h = inputs.Graph(g.n, g.row_ptr, g.col, g.row_ptr, g.col, w, w, True, "heavy")
    ref = _ref(h, 0)
    with ipg.Graph.from_inputs(h) as G:
        _check(G, ref, 0, policy="forced", forced_mode="pull", pr_engine="blocked")
        assert G.info()["bytes_blocked_layout"] == 0
        G.run("hashmin", policy="forced", forced_mode="pull", pr_engine="blocked")
        assert G.info()["bytes_blocked_layout"] > 0
        _check(G, ref, 0, policy="forced", forced_mode="pull", pr_engine="blocked")


def test_auto_builds_the_layout_for_sssp_after_enough_gather_pulls():
    g = inputs.rmat_graph(22, symmetrize=True, weighted=True, seed=2)
    assert g.m >= 1 << 26
    ref = _ref(g, 0)
    with ipg.Graph.from_inputs(g) as G:
        pulls, built_at = 0, None
        for run in range(8):
            st = _check(G, ref, 0, policy="forced", forced_mode="pull")
            if G.info()["bytes_blocked_layout"] and built_at is None:
                built_at = run
                assert pulls >= 6
            pulls += st.supersteps - 1
        assert built_at is not None


def test_vertex_count_times_weight_bound_keeps_the_gather():
    """V x the largest weight at or above 2^32 - 1: a distance plus a weight could reach
    the no-broadcast pattern, so SSSP keeps the gather pull (no layout is built for it)
    and stays exact. 2^24 + 70,000 vertices, most of them isolated, weights up to 255."""
    n = (1 << 24) + 70000
    core = inputs.rmat_graph(14, symmetrize=True, weighted=True, seed=12)
    assert int(core.w.max()) == 255 and n * 255 >= 0xFFFFFFFF
    row_ptr = np.concatenate([core.row_ptr, np.full(n - core.n, core.row_ptr[-1], np.uint32)])
    g = inputs.Graph(n, row_ptr, core.col, row_ptr, core.col, core.w, core.w, True, "sparse-wide")
    ref = _ref(g, 0)
    with ipg.Graph.from_inputs(g) as G:
        _check(G, ref, 0, policy="forced", forced_mode="pull", pr_engine="blocked")
        assert G.info()["bytes_blocked_layout"] == 0
