"""PageRank in forced pull through the CSC gather, run by the device-driven
superstep graph (one fused pull kernel and the selector per superstep, Fig. 8),
must give the same ranks, bit for bit, as the same exchange launched one kernel at
a time from the host (use_graph=0), the oracle's per-superstep counts, and the
oracle's ranks within 1e-5, on graphs in the caller's order and renumbered; the
superstep cap and T = 0 end a run early."""
import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2010_08781_gb300 as ipg  # noqa: E402

PULL = dict(policy="forced", forced_mode="pull", pr_engine="gather")


@pytest.mark.parametrize("name", ["rmat16", "rmat17", "star", "er_sinks", "cycle"])
def test_persistent_equals_host_loop_and_oracle(name):
    g = {
        "rmat16": lambda: inputs.rmat_graph(16, seed=1),  # the C1 configuration
        "rmat17": lambda: inputs.rmat_graph(17, seed=4),  # 1.9M edges: stored renumbered
        "star": lambda: inputs.star(20_000),  # a hub split into many chunks
        "er_sinks": lambda: inputs.from_edges(5000, *inputs.er_edges(2000, 20_000, seed=3)),
        "cycle": lambda: inputs.directed_cycle(777),
    }[name]()
    want, rst = oracle.pagerank(g.n, g.row_ptr, g.col, T=30)
    with ipg.Graph.from_inputs(g) as G:
        assert G.relabeled == (name == "rmat17")
        a = G.run("pagerank", **PULL)
        ra = G.values("pagerank")
        b = G.run("pagerank", use_graph=0, **PULL)
        rb = G.values("pagerank")
    assert np.array_equal(ra.view(np.uint32), rb.view(np.uint32))
    assert a.supersteps == b.supersteps == rst["supersteps"] and a.halted
    assert a.active.tolist() == rst["active"].tolist()
    assert a.messages.tolist() == rst["messages"].tolist()
    assert a.mode[1:].tolist() == [2] * (a.supersteps - 1)
    assert float(np.max(np.abs(ra.astype(np.float64) - want) / want)) <= 1e-5


def test_cap_and_zero_iterations():
    g = inputs.rmat_graph(12, seed=2)
    with ipg.Graph.from_inputs(g) as G:
        st = G.run("pagerank", max_supersteps=7, **PULL)
        assert st.code == ipg.IP_E_MAXSTEPS and st.supersteps == 7 and not st.halted
        capped = G.values("pagerank")
        want7, _ = oracle.pagerank(g.n, g.row_ptr, g.col, T=30, max_supersteps=7)
        assert float(np.max(np.abs(capped.astype(np.float64) - want7) / want7)) <= 1e-5
        st = G.run("pagerank", pr_iterations=0, **PULL)
        assert st.supersteps == 1 and st.halted
        assert np.allclose(G.values("pagerank"), 1.0 / g.n, rtol=1e-6)
        # repeated runs reuse the barrier and give the same bits
        G.run("pagerank", **PULL)
        r1 = G.values("pagerank")
        G.run("pagerank", **PULL)
        assert np.array_equal(r1.view(np.uint32), G.values("pagerank").view(np.uint32))
