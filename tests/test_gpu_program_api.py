"""The vertex-program interface (include/ipregel_program.cuh): an application the
paper does not have, the most reliable path, added as a program struct only
(csrc/app_reliability.cu) — FP32 values, a max combiner with no hardware atomic
(compare-and-swap loop) — against the oracle's run of the same program, bit for
bit (every product is one FP32 rounding on both sides and the max is exact) with
the per-superstep counts, in every exchange mode, under random mode sequences,
with the degree bins at their extremes (the CTA-chunk pull path combines partial
maxima across CTAs with the same CAS loop) and under the vertex renumbering.
Hashmin and SSSP run through the same engine in every other parity test."""
import ctypes

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
    st = G.run("reliability", **opts)
    got = G.values("reliability")
    want, rst = ref
    assert got.dtype == np.float32 and st.halted
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), int((got != want).sum())
    assert st.supersteps == rst["supersteps"]
    for k in ("active", "broadcasters", "messages"):
        assert getattr(st, k).tolist() == rst[k].tolist(), k
    return st


@pytest.fixture(scope="module")
def rel_graphs():
    return {
        "rmat12s_w": inputs.rmat_graph(12, symmetrize=True, weighted=True, seed=7),
        "rmat11d_w": inputs.rmat_graph(11, weighted=True, seed=8),
        "rmat12s_unit": inputs.rmat_graph(12, symmetrize=True, seed=9),
        "rmat12s_perm_w": inputs.rmat_graph(12, symmetrize=True, weighted=True, seed=7, permute_seed=5),
    }


@pytest.mark.parametrize("name", ["rmat12s_w", "rmat11d_w", "rmat12s_unit", "rmat12s_perm_w"])
@pytest.mark.parametrize("relabel", [False, True])
def test_reliability_every_mode(rel_graphs, name, relabel):
    g = rel_graphs[name]
    src = int(np.argmax(g.out_degree()))
    ref = oracle.reliability(g.n, g.row_ptr, g.col, g.w, source=src)
    with ipg.Graph.from_inputs(g, relabel=relabel) as G:
        for mode in ("push_sparse", "push_dense", "pull"):
            st = _check(G, ref, source=src, policy="forced", forced_mode=mode)
            assert all(m == ipg.MODES[mode] for m in st.mode[1:])
        _check(G, ref, source=src, policy="forced", forced_mode="pull", use_graph=0)
        for t1, t2 in ((1, 2), (64, 100000)):
            for mode in ("pull", "push_dense"):
                _check(G, ref, source=src, policy="forced", forced_mode=mode, t1=t1, t2=t2)
        rng = np.random.default_rng(3)
        _check(G, ref, source=src, mode_sequence=rng.integers(0, 3, 13).tolist())
        _check(G, ref, source=src, policy="threshold")


def test_reliability_sources_and_errors(rel_graphs):
    g = rel_graphs["rmat11d_w"]
    with ipg.Graph.from_inputs(g) as G:
        for src in (0, g.n - 1, int(np.argmin(g.out_degree()))):
            _check(G, oracle.reliability(g.n, g.row_ptr, g.col, g.w, source=src), source=src)
        with pytest.raises(ipg.IPError) as e:
            G.run("reliability", source=g.n)
        assert e.value.code == ipg.IP_E_RANGE
        # an application id no program registered
        o = ipg.default_options()
        code = ipg.load().ip_run(G._h, 7, 100, ctypes.byref(o), None)
        assert code == ipg.IP_E_INVAL
