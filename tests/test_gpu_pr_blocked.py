"""Blocked PageRank pull (IP_PR_ENGINE_BLOCKED) against the FP64 oracle.

The blocked engine computes the same PULL exchange as the CSC gather (every
vertex sums its in-neighbours' broadcasts, Fig. 8) through a second edge layout:
runs of entries from a chunk of sources into a bin of destinations, the sources'
broadcasts written next to the entries as fixed-point codes, and every bin summed
exactly in shared memory. The bar is the one of every PageRank path: max relative
error 1e-5 per vertex of the FP64 oracle. The graphs below reach every structural
case of the layout: a single source with more out-edges than a chunk's target (a
chunk of one source), a destination with more in-edges than a bin's target (a bin
of few vertices), runs padded to 4 entries, chunks cut by their source count,
long stretches of sources without out-edges, partial bins, codes of 2^31 units or
more (the high word of the sums), and mode sequences that switch between the
blocked pull and the push exchange (broadcasts rebuilt from ranks).
"""
import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2010_08781_gb300 as ipg  # noqa: E402

PR_RTOL = 1e-5


def _ref(g, T=30):
    return oracle.pagerank(g.n, g.row_ptr, g.col, T=T, damping=0.85)


def _err(got, want):
    return float(np.max(np.abs(got.astype(np.float64) - want) / np.abs(want)))


def _blocked(G, **kw):
    kw.setdefault("policy", "forced")
    kw.setdefault("forced_mode", "pull")
    st = G.run("pagerank", pr_engine="blocked", **kw)
    return st, G.values("pagerank")


def _hub_graph():
    """An out-hub of 300,000 edges (a chunk of one source, long runs), an in-hub of
    1.2M edges (a bin of few vertices), sources without out-edges, and an ER
    background."""
    n = 1_300_000
    rng = np.random.default_rng(7)
    out_src = np.zeros(300_000, np.uint32)
    out_dst = np.arange(1, 300_001, dtype=np.uint32)
    in_src = np.arange(100_000, 1_300_000, dtype=np.uint32)
    in_dst = np.full(in_src.shape, 5, np.uint32)
    bs = rng.integers(0, 600_000, 2_000_000).astype(np.uint32)  # sources >= 600,000 only point at the hub
    bd = rng.integers(0, n, 2_000_000).astype(np.uint32)
    return inputs.from_edges(n, np.concatenate([out_src, in_src, bs]), np.concatenate([out_dst, in_dst, bd]))


@pytest.mark.parametrize("name", ["cycle", "complete", "star", "path", "selfloops", "er", "rmat12", "rmat11s",
                                  "isolated"])
def test_small_graphs(name):
    g = {
        "cycle": lambda: inputs.directed_cycle(65),
        "complete": lambda: inputs.complete_digraph(40),
        "star": lambda: inputs.star(300),
        "path": lambda: inputs.path(33),
        "selfloops": lambda: inputs.from_edges(3, [0, 1, 1, 2], [0, 1, 2, 2]),
        "er": lambda: inputs.er_graph(3000, 9000, seed=4),
        "rmat12": lambda: inputs.rmat_graph(12, seed=5),
        "rmat11s": lambda: inputs.rmat_graph(11, symmetrize=True, seed=6),
        # 40,000 vertices of which only the first 50 have out-edges: long runs of
        # sources without out-edges, and a second, partial bin
        "isolated": lambda: inputs.from_edges(40_000, np.arange(50, dtype=np.uint32) % 50,
                                              (np.arange(50, dtype=np.uint32) * 797) % 40_000),
    }[name]()
    want, rst = _ref(g)
    with ipg.Graph.from_inputs(g) as G:
        st, got = _blocked(G)
    assert st.supersteps == rst["supersteps"]
    assert _err(got, want) <= PR_RTOL


def test_closed_forms():
    """Directed cycle and complete digraph: every iterate is 1/N. Star: the exact
    finite-T iterate derived from the two-state recurrence."""
    for g in (inputs.directed_cycle(1000), inputs.complete_digraph(64)):
        with ipg.Graph.from_inputs(g) as G:
            _, r = _blocked(G)
        assert np.max(np.abs(r.astype(np.float64) * g.n - 1.0)) <= PR_RTOL
    k, d = 50_000, 0.85  # the centre's 50,000 out-edges: runs of one chunk into three bins
    N = k + 1
    rc = (1 + d * k) / (N * (1 + d))
    rl = (1 - d) / N + d * rc / k
    ec, el = 1.0 / N - rc, 1.0 / N - rl
    for _ in range(30):
        ec, el = d * k * el, d * ec / k
    with ipg.Graph.from_inputs(inputs.star(k)) as G:
        _, r = _blocked(G)
    r = r.astype(np.float64)
    assert abs(r[0] - (rc + ec)) / (rc + ec) <= PR_RTOL
    assert np.max(np.abs(r[1:] - (rl + el)) / (rl + el)) <= PR_RTOL


def test_scale16_config_and_engines_agree():
    g = inputs.rmat_graph(16, seed=1)  # directed R-MAT scale 16, edge factor 16, seed 1
    want, rst = _ref(g)
    with ipg.Graph.from_inputs(g) as G:
        st, got = _blocked(G)
        G.run("pagerank", policy="forced", forced_mode="pull", pr_engine="gather")
        gat = G.values("pagerank")
    assert st.active.tolist() == rst["active"].tolist()
    assert st.messages.tolist() == rst["messages"].tolist()
    assert _err(got, want) <= PR_RTOL
    assert _err(gat, want) <= PR_RTOL


def test_hubs_split_bins_and_long_runs():
    g = _hub_graph()
    want, _ = _ref(g)
    with ipg.Graph.from_inputs(g) as G:
        _, got = _blocked(G)
    assert _err(got, want) <= PR_RTOL


def test_rmat20_and_determinism():
    g = inputs.rmat_graph(20, seed=1)  # 16M edges: hundreds of chunks and bins
    want, _ = _ref(g)
    with ipg.Graph.from_inputs(g) as G:
        _, a = _blocked(G)
        _, b = _blocked(G, use_graph=0)
        _, c = _blocked(G, profile_kernels=1)
    assert _err(a, want) <= PR_RTOL
    # the fixed-point sums do not depend on the order of the additions
    assert np.array_equal(a, b) and np.array_equal(a, c)


def test_rmat22_thirty_updates_against_the_oracle():
    """The whole T = 30 trajectory at R-MAT 22 (65M edges: the engine AUTO picks from
    2^24 edges, renumbered, over a thousand chunks and bins) against the FP64
    oracle's 30 updates, every vertex: the fixed-point sums keep the per-vertex
    error within the bar after 30 rounds of feeding the engine's own ranks back."""
    g = inputs.rmat_graph(22, seed=1)
    want, _ = _ref(g)
    with ipg.Graph.from_inputs(g) as G:
        st = G.run("pagerank")  # AUTO engine, default policy: the configuration the bench times
        got = G.values("pagerank")
        assert st.supersteps == 31
        assert G.info()["bytes_blocked_layout"] > 0  # the blocked engine ran
    assert _err(got, want) <= PR_RTOL
    assert abs(float(np.sum(got.astype(np.float64))) - float(np.sum(want))) <= 1e-4


def test_mode_sequences_and_auto_policy():
    g = inputs.rmat_graph(14, seed=3)
    want, _ = _ref(g)
    with ipg.Graph.from_inputs(g) as G:
        for seq in (["pull", "push_dense"], ["push_dense", "pull", "pull"]):
            _, got = _blocked(G, mode_sequence=seq, policy="sequence")
            assert _err(got, want) <= PR_RTOL
        G.run("pagerank", pr_engine="blocked")
        assert _err(G.values("pagerank"), want) <= PR_RTOL
        _, t10 = _blocked(G, pr_iterations=10)
    want10, _ = _ref(g, T=10)
    assert _err(t10, want10) <= PR_RTOL


def test_unsupported_and_invalid():
    with ipg.Graph.from_inputs(inputs.empty_graph(10)) as G:
        with pytest.raises(ipg.IPError) as ei:
            G.run("pagerank", pr_engine="blocked", policy="forced", forced_mode="pull")
        assert ei.value.code == ipg.IP_E_RANGE
        G.run("pagerank", policy="forced", forced_mode="pull")  # AUTO picks the gather engine here
        assert np.allclose(G.values("pagerank"), 0.15 / 10, rtol=PR_RTOL)
        with pytest.raises(ipg.IPError) as ei:
            G.run("pagerank", pr_engine=7)
        assert ei.value.code == ipg.IP_E_INVAL
