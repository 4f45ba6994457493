"""Graph creation from page-locked host arrays: such arrays are read by the
device directly (a copy kernel that also checks the vertex ids, or, when the
graph is renumbered during creation, the renumbering copy itself, which checks
them too), every other host array by a DMA copy. Both routes must build the same graph: results against
the oracle for CSR-only, CSR + CSC and symmetric inputs with edge counts that are
not multiples of 4, a misaligned page-locked view (DMA route), and an
out-of-range id or a decreasing offset refused with the same codes as the check
kernels of the other route."""
import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2010_08781_gb300 as ipg  # noqa: E402


def _pin(a, offset=0):
    """A page-locked int32 copy of a uint32 array; offset > 0 returns a view that
    starts `offset` words into a larger page-locked buffer (4-byte aligned only)."""
    a = np.ascontiguousarray(a, dtype=np.uint32)
    t = torch.empty(a.size + offset, dtype=torch.int32, pin_memory=True)
    t[offset:] = torch.from_numpy(a.view(np.int32))
    return t[offset:]


@pytest.mark.parametrize("relabel", [False, True])
@pytest.mark.parametrize("offset", [0, 1])
def test_pinned_inputs_build_the_same_graph(offset, relabel):
    g = inputs.rmat_graph(11, symmetrize=True, weighted=True, seed=3)
    assert g.m % 4 != 0 or offset
    ref = {"hashmin": oracle.hashmin(g.n, g.row_ptr, g.col)[0], "sssp": oracle.sssp(g.n, g.row_ptr, g.col, g.w)[0]}
    p = [_pin(x, offset) for x in (g.row_ptr, g.col, g.w)]
    assert p[1].is_pinned()
    with ipg.Graph(g.n, p[0], p[1], p[2], symmetric=True, relabel=relabel) as G:
        for app in ("hashmin", "sssp"):
            G.run(app)
            assert np.array_equal(G.values(app), ref[app]), app
    d = inputs.rmat_graph(10, seed=4)
    want, _ = oracle.pagerank(d.n, d.row_ptr, d.col, T=30)
    for csc in (False, True):
        arrs = [_pin(d.row_ptr, offset), _pin(d.col, offset)]
        kw = dict(csc_offsets=_pin(d.t_ptr, offset), csc_rows=_pin(d.t_idx, offset)) if csc else {}
        with ipg.Graph(d.n, *arrs, relabel=relabel, **kw) as G:
            G.run("pagerank")
            got = G.values("pagerank").astype(np.float64)
        assert float(np.max(np.abs(got - want) / want)) <= 1e-5


@pytest.mark.parametrize("relabel", [False, True])
@pytest.mark.parametrize("offset", [0, 1])
def test_pinned_inputs_are_checked(offset, relabel):
    g = inputs.rmat_graph(10, symmetrize=True, seed=5)
    col = g.col.copy()
    col[-1] = g.n + 3  # the last word: the copy kernel's tail when E is not a multiple of 4
    col[len(col) // 3] = g.n
    with pytest.raises(ipg.IPError) as e:
        ipg.Graph(g.n, _pin(g.row_ptr, offset), _pin(col, offset), symmetric=True, relabel=relabel)
    assert e.value.code == ipg.IP_E_RANGE
    off = g.row_ptr.copy()
    off[5] = off[6] + 1  # decreasing
    with pytest.raises(ipg.IPError) as e:
        ipg.Graph(g.n, _pin(off, offset), _pin(g.col, offset), symmetric=True, relabel=relabel)
    assert e.value.code == ipg.IP_E_INVAL
    with ipg.Graph(g.n, _pin(g.row_ptr, offset), _pin(g.col, offset), symmetric=True,
                   relabel=relabel) as G:  # and then a good one
        G.run("hashmin")
        assert np.array_equal(G.values("hashmin"), oracle.hashmin(g.n, g.row_ptr, g.col)[0])


@pytest.mark.parametrize("relabel", [False, True])
def test_in_edge_rows_wait_for_the_first_run_that_reads_them(relabel):
    """A directed graph created without a CSC holds the transpose's offsets only. The
    blocked pull (PageRank, SSSP) streams its own layout and leaves it so; the first
    run that reads in-edge rows (a pull on the gather engine, a batched run) builds
    them, weights included, and every result matches the oracle."""
    d = inputs.rmat_graph(12, weighted=True, seed=6)
    ea = ((d.m + 3) // 4) * 4 + 4
    pr, _ = oracle.pagerank(d.n, d.row_ptr, d.col, T=30)
    srcs = [0, 5, 77]
    ss = [oracle.sssp(d.n, d.row_ptr, d.col, d.w, source=s)[0] for s in srcs]
    with ipg.Graph(d.n, d.row_ptr, d.col, d.w, relabel=relabel) as G:
        csr = (d.n + 1) * 4 + 2 * ea * 4
        assert G.info()["bytes_graph"] == csr + (d.n + 1) * 4
        G.run("pagerank", policy="forced", forced_mode="pull", pr_engine="blocked")
        got = G.values("pagerank").astype(np.float64)
        assert float(np.max(np.abs(got - pr) / pr)) <= 1e-5
        assert G.info()["bytes_graph"] == csr + (d.n + 1) * 4
        G.run("sssp", source=srcs[1], policy="forced", forced_mode="pull", pr_engine="blocked")
        assert np.array_equal(G.values("sssp"), ss[1])
        assert G.info()["bytes_graph"] == csr + (d.n + 1) * 4
        G.run("sssp", source=srcs[0], policy="forced", forced_mode="pull", pr_engine="gather")
        assert np.array_equal(G.values("sssp"), ss[0])
        assert G.info()["bytes_graph"] == 2 * csr
        G.run("pagerank", policy="forced", forced_mode="pull", pr_engine="gather")
        got = G.values("pagerank").astype(np.float64)
        assert float(np.max(np.abs(got - pr) / pr)) <= 1e-5
    with ipg.Graph(d.n, d.row_ptr, d.col, d.w, relabel=relabel) as G:  # a batched run first
        dist, _ = G.run_batch_sssp(srcs)
        for i in range(len(srcs)):
            assert np.array_equal(dist[i], ss[i]), i
        assert G.info()["bytes_graph"] == 2 * csr


@pytest.mark.parametrize("offset", [0, 1])
def test_pinned_directed_weighted_renumbered(offset):
    """Directed weighted graph from page-locked arrays, renumbered during creation:
    the renumbering copy reads columns and weights from the host and counts the
    in-degrees on the way (offset 0), or the arrays are copied first (offset 1, a
    view the copy kernel cannot read at 16-byte alignment); SSSP on both pull engines,
    PageRank and the in-degree maximum match the oracle."""
    d = inputs.rmat_graph(12, weighted=True, seed=13)
    ss, _ = oracle.sssp(d.n, d.row_ptr, d.col, d.w, source=3)
    pr, _ = oracle.pagerank(d.n, d.row_ptr, d.col, T=30)
    with ipg.Graph(d.n, _pin(d.row_ptr, offset), _pin(d.col, offset), _pin(d.w, offset), relabel=True) as G:
        assert G.info()["max_in_degree"] == int(np.diff(d.t_ptr.astype(np.int64)).max())
        for eng in ("gather", "blocked"):
            G.run("sssp", source=3, policy="forced", forced_mode="pull", pr_engine=eng)
            assert np.array_equal(G.values("sssp"), ss), eng
        G.run("pagerank", policy="forced", forced_mode="pull")
        got = G.values("pagerank").astype(np.float64)
        assert float(np.max(np.abs(got - pr) / pr)) <= 1e-5
