"""PageRank to convergence on the GPU (ip_options_t.pr_tolerance) against the
oracle's convergence rule: the run ends after the first superstep s >= 1 whose
L1 rank change sum_v |r_s(v) - r_(s-1)(v)| is below the tolerance, T still
capping it. Both sides must stop at the same superstep and the ranks must agree
within 1e-5 relative per vertex. The tolerances sit between two consecutive
changes of the oracle's run (their geometric mean), far from either, so the FP32
change of the GPU cannot fall on the other side of the tolerance."""
import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2010_08781_gb300 as ipg  # noqa: E402

RTOL = 1e-5
MODES = [dict(policy="forced", forced_mode="pull", pr_engine="gather"),
         dict(policy="forced", forced_mode="pull", pr_engine="blocked"),
         dict(policy="forced", forced_mode="push_dense"),
         dict(policy="forced", forced_mode="pull", pr_engine="blocked", use_graph=0)]


def _between(delta, t):
    """A tolerance between the changes of supersteps t - 1 and t (float32-exact)."""
    eps = np.float32(np.sqrt(delta[t] * delta[t - 1]))
    assert delta[t] < eps < delta[t - 1] and min(eps / delta[t], delta[t - 1] / eps) > 1.01
    return float(eps)


@pytest.mark.parametrize("kw", MODES, ids=["gather", "blocked", "push", "blocked_host_loop"])
@pytest.mark.parametrize("name", ["rmat14", "rmat12_sym"])
def test_convergence_halts_where_the_oracle_does(name, kw):
    g = inputs.rmat_graph(14, seed=6) if name == "rmat14" else inputs.rmat_graph(12, symmetrize=True, seed=6)
    _, full = oracle.pagerank(g.n, g.row_ptr, g.col, T=60)
    for t_halt in (4, 11):
        eps = _between(full["delta"], t_halt)
        want, ost = oracle.pagerank(g.n, g.row_ptr, g.col, T=60, tolerance=eps)
        assert ost["supersteps"] == t_halt + 1
        with ipg.Graph.from_inputs(g, relabel=False) as G:
            st = G.run("pagerank", pr_iterations=60, pr_tolerance=eps, **kw)
            got = G.values("pagerank").astype(np.float64)
        assert st.halted and st.supersteps == ost["supersteps"], (st.supersteps, ost["supersteps"])
        err = np.abs(got - want) / want
        assert float(err.max()) <= RTOL, float(err.max())
        # the GPU's own L1 changes, superstep by superstep: its FP32 ranks carry about
        # 1e-7 relative error each, so the change carries about 1e-7 (sum of the ranks <= 1)
        np.testing.assert_allclose(st.pr_delta[1:t_halt + 1], ost["delta"][1:t_halt + 1], rtol=1e-3, atol=5e-7)


def test_convergence_closed_forms_and_cap():
    """Directed cycle: the first update changes nothing (halt after superstep 1).
    Star: the halting superstep of the closed form. A cap T below the halting
    superstep stops the run at T, and without a tolerance no change is recorded."""
    cyc = inputs.directed_cycle(64)
    with ipg.Graph.from_inputs(cyc) as G:
        st = G.run("pagerank", pr_iterations=30, pr_tolerance=1e-9)
        assert st.halted and st.supersteps == 2
        np.testing.assert_allclose(G.values("pagerank"), 1.0 / 64, rtol=RTOL)
    k, d = 40, 0.85
    star = inputs.star(k)
    _, full = oracle.pagerank(star.n, star.row_ptr, star.col, T=120)
    eps = _between(full["delta"], 30)
    want, ost = oracle.pagerank(star.n, star.row_ptr, star.col, T=120, tolerance=eps)
    with ipg.Graph.from_inputs(star) as G:
        st = G.run("pagerank", pr_iterations=120, pr_tolerance=eps)
        assert st.supersteps == ost["supersteps"] == 31
        assert float(np.max(np.abs(G.values("pagerank") - want) / want)) <= RTOL
        st = G.run("pagerank", pr_iterations=10, pr_tolerance=eps)  # T first
        assert st.halted and st.supersteps == 11
        st = G.run("pagerank", pr_iterations=10)
        assert st.supersteps == 11 and not st.pr_delta.any()


def test_convergence_rejects_bad_tolerance():
    g = inputs.directed_cycle(8)
    with ipg.Graph.from_inputs(g) as G:
        for bad in (-1.0, float("nan")):
            with pytest.raises(ipg.IPError) as e:
                G.run("pagerank", pr_tolerance=bad)
            assert e.value.code == ipg.IP_E_INVAL
