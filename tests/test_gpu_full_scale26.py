"""The billion-edge configuration at full size (R-MAT scale 26, edge factor 16,
(a, b, c) = (.57, .19, .19), seed 1: 67,108,864 vertices, 1,060,392,804 directed
edges), in the launch configuration the benchmark times: the graph handed over
as page-locked host CSR (the end-to-end path: the renumbering copy reads the edges
over the host link itself, checks them, and counts the in-degrees on the way),
vertices renumbered by degree class, PageRank in forced pull with the AUTO engine
(the blocked pull here).

PageRank: a full FP64 oracle run takes about 11 s per superstep on one core, so
the last superstep is checked one vertex at a time instead. With the ranks of a
run of T - 1 = 29 iterations, ``oracle.pagerank_update`` computes superstep 30 of
Fig. 8 for a sample of vertices (the 64 largest in-degrees, vertices without
in-edges, vertices without out-edges, random vertices), which
must match the T = 30 run within 1e-5 relative; every rank must be at least
(1 - d)/N. Hashmin on the symmetrised graph (2.1 billion directed edges): every
label against a full oracle run (Fig. 9)."""
import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2010_08781_gb300 as ipg  # noqa: E402

SCALE = 26
PR_RTOL = 1e-5


def _pinned(a):
    """A page-locked int32 copy of a uint32 array."""
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).pin_memory()


@pytest.fixture(scope="module")
def edges():
    return inputs.rmat_edges(SCALE, 16 << SCALE, 0.57, 0.19, 0.19, 1)


def test_pagerank_last_superstep_sampled(edges):
    g = inputs.from_edges(1 << SCALE, edges[0], edges[1])
    n, d = g.n, 0.85
    kw = dict(policy="forced", forced_mode="pull")
    with ipg.Graph(n, _pinned(g.row_ptr), _pinned(g.col)) as G:
        assert G.relabeled
        st29 = G.run("pagerank", pr_iterations=29, **kw)
        r29 = G.values("pagerank").astype(np.float64)
        st30 = G.run("pagerank", pr_iterations=30, **kw)
        r30 = G.values("pagerank").astype(np.float64)
    assert st29.halted and st30.halted and st30.supersteps == 31
    assert st30.messages[:30].tolist() == [g.m] * 30
    indeg = np.diff(g.t_ptr.astype(np.int64))
    outdeg = g.out_degree()
    rng = np.random.default_rng(26)
    pick = np.unique(np.concatenate([
        np.argsort(indeg)[-64:],                            # the largest in-degrees
        np.flatnonzero(indeg == 0)[:64],                    # rank (1 - d)/N exactly
        np.flatnonzero((indeg > 0) & (outdeg == 0))[:64],   # vertices without out-edges
        rng.integers(0, n, 2048),
    ])).astype(np.int64)
    want = oracle.pagerank_update(pick, n, g.t_ptr, g.t_idx, outdeg, r29, damping=d)
    err = np.abs(r30[pick] - want) / want
    assert float(err.max()) <= PR_RTOL, (int(pick[np.argmax(err)]), float(err.max()))
    assert float(r30.min()) >= (1 - d) / n * (1 - PR_RTOL)


def test_hashmin_every_label(edges):
    gs = inputs.from_edges(1 << SCALE, edges[0], edges[1], symmetrize=True)
    ptr, col = _pinned(gs.row_ptr), _pinned(gs.col)
    with ipg.Graph(gs.n, ptr, col, symmetric=True) as G:
        st = G.run("hashmin")
        got = G.values("hashmin")
    want, ost = oracle.hashmin(gs.n, gs.row_ptr, gs.col)
    assert np.array_equal(got, want), int((got != want).sum())
    assert st.halted and st.supersteps == ost["supersteps"]
    for k in ("active", "broadcasters", "messages"):
        assert getattr(st, k).tolist() == ost[k].tolist(), k
