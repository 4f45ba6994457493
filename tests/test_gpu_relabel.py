"""Vertex renumbering inside the handle (ip_graph_relabel): the library stores the
graph with its vertices ordered by out-degree class, and every result must still be
the one of the graph as the caller numbered it, bit for bit for Hashmin and SSSP
(labels are the smallest CALLER id of each component, Fig. 9; distances from the
caller's source, Fig. 10) and within 1e-5 of the FP64 oracle for PageRank (Fig. 8).
The graphs reach every case of the renumbering: a symmetric graph (one shared
edge store), a directed graph whose in-edges are transposed again, hubs that move
to the front, vertices without out-edges that move to the back, and batched runs
whose sources and instance ranges are given in the caller's numbering."""
import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2010_08781_gb300 as ipg  # noqa: E402

MODES = ("push_sparse", "push_dense", "pull")


def _graphs():
    # a star whose centre is the LAST caller id: after renumbering it comes first,
    # so a Hashmin run that labelled by internal id would answer with the centre
    k = 500
    star_last = inputs.from_edges(k + 1, np.full(k, k, np.uint32), np.arange(k, dtype=np.uint32), symmetrize=True,
                                  weighted=True)
    # a third of the vertices without out-edges, spread over the id range
    rng = np.random.default_rng(11)
    n = 6000
    src = rng.integers(0, n, 30_000).astype(np.uint32)
    src = src[src % 3 != 1]
    dst = rng.integers(0, n, src.size).astype(np.uint32)
    return {
        "rmat12_sym_w": inputs.rmat_graph(12, symmetrize=True, weighted=True, seed=21),
        "rmat12_dir_w": inputs.rmat_graph(12, weighted=True, seed=22),
        "star_last": star_last,
        "sinks_dir": inputs.from_edges(n, src, dst, weighted=True),
    }


GRAPHS = _graphs()


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_every_app_and_mode_in_caller_numbering(name):
    g = GRAPHS[name]
    hm, hst = oracle.hashmin(g.n, g.row_ptr, g.col)
    pr, _ = oracle.pagerank(g.n, g.row_ptr, g.col)
    deg = np.diff(g.row_ptr.astype(np.int64))
    sources = [0, g.n - 1, int(np.argmax(deg)), int(np.argmin(deg))]
    with ipg.Graph.from_inputs(g, relabel=True) as G:
        assert G.relabeled
        for mode in MODES:
            st = G.run("hashmin", policy="forced", forced_mode=mode)
            assert np.array_equal(G.values("hashmin"), hm), mode
            assert st.supersteps == hst["supersteps"]
            for s in sources:
                want, sst = oracle.sssp(g.n, g.row_ptr, g.col, g.w, source=s)
                st = G.run("sssp", source=s, policy="forced", forced_mode=mode)
                assert np.array_equal(G.values("sssp"), want), (mode, s)
                assert st.supersteps == sst["supersteps"]
        G.run("hashmin")
        assert np.array_equal(G.values("hashmin"), hm)
        for eng in ("gather", "blocked"):
            G.run("pagerank", policy="forced", forced_mode="pull", pr_engine=eng)
            r = G.values("pagerank").astype(np.float64)
            assert np.max(np.abs(r - pr) / pr) <= 1e-5, eng
        G.run("pagerank", mode_sequence=["push_dense", "pull"], policy="sequence")
        r = G.values("pagerank").astype(np.float64)
        assert np.max(np.abs(r - pr) / pr) <= 1e-5


def test_build_csc_on_device_and_device_output():
    g = inputs.rmat_graph(13, weighted=True, seed=23)
    want, _ = oracle.sssp(g.n, g.row_ptr, g.col, g.w, source=5)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    with ipg.Graph.from_inputs(g, build_csc_on_device=True, relabel=True) as G:
        G.run("sssp", source=5, policy="forced", forced_mode="pull")
        G.values(out=out)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), want)


def test_state_rules():
    g = inputs.rmat_graph(11, symmetrize=True, seed=24)
    hm, _ = oracle.hashmin(g.n, g.row_ptr, g.col)
    with ipg.Graph.from_inputs(g, relabel=False) as G:
        G.run("hashmin")
        G.relabel()  # drops the values of the run before it
        with pytest.raises(ipg.IPError) as ei:
            G.values("hashmin")
        assert ei.value.code == ipg.IP_E_STATE
        G.relabel()  # a second call changes nothing
        G.run("hashmin")
        assert np.array_equal(G.values("hashmin"), hm)


def test_auto_threshold():
    small = inputs.rmat_graph(10, symmetrize=True, seed=25)
    big = inputs.rmat_graph(17, seed=26)  # 1.9M directed edges
    assert big.m >= ipg.RELABEL_AUTO_EDGES > small.m
    with ipg.Graph.from_inputs(small) as G:
        assert not G.relabeled
    want, _ = oracle.sssp(big.n, big.row_ptr, big.col, big.w, source=3)
    with ipg.Graph.from_inputs(big) as G:
        assert G.relabeled
        G.run("sssp", source=3)
        assert np.array_equal(G.values("sssp"), want)


def test_batched_sssp():
    g = inputs.rmat_graph(11, symmetrize=True, weighted=True, seed=27)
    sources = np.concatenate([[0, g.n - 1], inputs.uniform_vertices(g.n, 38, seed=3)]).astype(np.uint32)
    with ipg.Graph.from_inputs(g, relabel=True) as G:
        dist, st = G.run_batch_sssp(sources)
    for i, s in enumerate(sources):
        want, ost = oracle.sssp(g.n, g.row_ptr, g.col, g.w, source=int(s))
        assert np.array_equal(dist[i], want), s
        assert st["instance_supersteps"][i] == ost["supersteps"], s


@pytest.mark.parametrize("engine", ["graph", "persistent"])
def test_batched_hashmin(engine):
    rng = np.random.default_rng(8)
    gs = [inputs.rmat_sized(int(n), 8, seed=200 + i) for i, n in enumerate(rng.integers(1, 2500, 20))]
    gs.append(inputs.empty_graph(5))
    u, offs = inputs.block_diagonal(gs)
    with ipg.Graph.from_inputs(u, relabel=True) as G:
        labels, st = G.run_batch_hashmin(offs.astype(np.uint32), engine=engine)
    assert st["halted"]
    for i, h in enumerate(gs):
        want, ost = oracle.hashmin(h.n, h.row_ptr, h.col)
        assert np.array_equal(labels[offs[i]:offs[i + 1]], want), i
        assert st["instance_supersteps"][i] == ost["supersteps"], i
