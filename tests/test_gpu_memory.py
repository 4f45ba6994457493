"""The library's device-buffer cache: graphs destroyed and created again with the
same shape reuse buffers that still hold the previous graph's data, so every
result must not depend on what a buffer held before (the apps run in every mode
on graphs of identical sizes but different edges), and releasing the cache must
leave the library usable."""
import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2010_08781_gb300 as ipg  # noqa: E402


def _relabel(g, seed):
    """The same graph under a random vertex permutation: identical buffer sizes, other contents."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(g.n).astype(np.uint32)
    src = np.repeat(np.arange(g.n, dtype=np.uint32), np.diff(g.row_ptr.astype(np.int64)))
    return inputs.from_edges(g.n, perm[src], perm[g.col], symmetrize=g.symmetric, weighted=g.w is not None)


def test_reused_buffers_give_the_same_results():
    base = inputs.rmat_graph(13, symmetrize=True, weighted=True, seed=2)
    graphs = [base, _relabel(base, 1), _relabel(base, 2), base]
    for g in graphs:
        hm, _ = oracle.hashmin(g.n, g.row_ptr, g.col)
        ss, _ = oracle.sssp(g.n, g.row_ptr, g.col, g.w, source=0)
        pr, _ = oracle.pagerank(g.n, g.row_ptr, g.col)
        with ipg.Graph.from_inputs(g) as G:
            for mode in ("push_sparse", "push_dense", "pull"):
                G.run("hashmin", policy="forced", forced_mode=mode)
                assert np.array_equal(G.values("hashmin"), hm)
                G.run("sssp", policy="forced", forced_mode=mode)
                assert np.array_equal(G.values("sssp"), ss)
            for eng in ("gather", "blocked"):
                G.run("pagerank", policy="forced", forced_mode="pull", pr_engine=eng)
                r = G.values("pagerank").astype(np.float64)
                assert np.max(np.abs(r - pr) / pr) <= 1e-5


def test_release_cached_memory_then_create():
    g = inputs.rmat_graph(12, symmetrize=True, weighted=True, seed=3)
    want, _ = oracle.sssp(g.n, g.row_ptr, g.col, g.w, source=0)
    for _ in range(2):
        with ipg.Graph.from_inputs(g) as G:
            G.run("sssp")
            assert np.array_equal(G.values("sssp"), want)
        ipg.release_cached_memory()


def test_memory_footprint_breakdown():
    """ip_graph_info's parts add up to the handle's device bytes and each part has
    its expected size: graph store, 13 vertex arrays plus 3 bitmaps, the two maps
    of the renumbering, and the blocked layout once a blocked pull has run."""
    d = inputs.rmat_graph(14, seed=3)
    with ipg.Graph(d.n, d.row_ptr, d.col, relabel=True) as G:
        i0 = G.info()
        n, ea = d.n, ((d.m + 3) // 4) * 4 + 4
        # CSR and the device-built transpose's offsets: its rows wait for a run that reads them
        assert i0["bytes_graph"] == 2 * (n + 1) * 4 + ea * 4
        words = ((n + 31) // 32 + 31) // 32 * 32
        assert i0["bytes_vertex_state"] >= 13 * n * 4 + 3 * words * 4
        assert i0["bytes_renumbering"] == 8 * n
        assert i0["bytes_degree_bins"] > 0 and i0["bytes_blocked_layout"] == 0
        G.run("pagerank", policy="forced", forced_mode="pull", pr_engine="blocked")
        i1 = G.info()
        assert i1["bytes_blocked_layout"] >= 8 * d.m  # about 8 bytes per edge
        assert i1["bytes_graph"] == i0["bytes_graph"]  # the blocked pull reads no in-edge rows
        G.run("hashmin", policy="forced", forced_mode="pull")
        i2 = G.info()
        assert i2["bytes_graph"] == 2 * ((n + 1) * 4 + ea * 4)  # the gather pull built them
        for info in (i0, i1, i2):
            parts = sum(info[k] for k in info if k.startswith("bytes_"))
            assert parts == info["device_bytes"]
            assert info["bytes_other"] < 1 << 23  # run log (up to 65,536 supersteps), selector, control
    s = inputs.rmat_graph(12, symmetrize=True, weighted=True, seed=3)
    with ipg.Graph.from_inputs(s, relabel=False) as G:
        info = G.info()
        assert info["bytes_graph"] == (s.n + 1) * 4 + 2 * (((s.m + 3) // 4) * 4 + 4) * 4  # shared CSR/CSC, weights
        assert info["bytes_renumbering"] == 0
