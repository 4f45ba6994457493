"""The allocation-free Hashmin entry point (ip_hashmin_noalloc) against ip_run.

Some callers cannot allocate device memory (they run inside another
framework's memory pool or under a fixed budget); this entry point keeps its
temporary state in a fixed array inside the library. The test calls it twice
in a row through the C ABI, on graphs of different sizes, so the second call
also checks that state left behind by the first is cleared, and compares the
labels and the superstep count with ip_run's Hashmin (bit-exact: integer labels).
"""
import numpy as np
import pytest

import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2010_08781_gb300 as ipg  # noqa: E402


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def test_noalloc_hashmin_matches_ip_run_twice():
    graphs = [inputs.rmat_graph(14, symmetrize=True, seed=3), inputs.rmat_graph(12, seed=4)]
    for g in graphs:  # two calls in a row, different sizes
        with ipg.Graph.from_inputs(g) as G:
            st = G.run("hashmin", policy="threshold")
            want = G.values("hashmin")
        labels = torch.full((g.n,), -1, dtype=torch.int32, device="cuda")
        code, steps = ipg.hashmin_noalloc(g.n, _dev(g.row_ptr), _dev(g.col), labels)
        assert code == ipg.IP_OK
        assert steps == st.supersteps
        assert np.array_equal(labels.cpu().numpy().view(np.uint32), want)


def test_noalloc_rejects_oversized_graph():
    off = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    code, _ = ipg.hashmin_noalloc(ipg.NOALLOC_MAX_VERTICES + 1, off, off, out)
    assert code == ipg.IP_E_RANGE


def test_noalloc_checks_its_input_then_runs_clean():
    """Malformed graphs are refused by the entry point's own device checks (no
    access leaves the arrays), and a valid call right after still matches ip_run."""
    g = inputs.rmat_graph(10, symmetrize=True, seed=5)
    out = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    bad_col = g.col.copy()
    bad_col[len(bad_col) // 2] = g.n + 7  # a destination beyond the last vertex
    code, _ = ipg.hashmin_noalloc(g.n, _dev(g.row_ptr), _dev(bad_col), out)
    assert code == ipg.IP_E_RANGE
    bad_off = g.row_ptr.copy()
    assert bad_off[3] > 0
    bad_off[4] = bad_off[3] - 1  # a decreasing pair of offsets
    code, _ = ipg.hashmin_noalloc(g.n, _dev(bad_off), _dev(g.col), out)
    assert code == ipg.IP_E_INVAL
    short = g.row_ptr.copy()
    short[-1] -= 1  # the last offset is not n_edges
    code, _ = ipg.hashmin_noalloc(g.n, _dev(short), _dev(g.col), out)
    assert code == ipg.IP_E_INVAL
    with ipg.Graph.from_inputs(g) as G:
        st = G.run("hashmin", policy="threshold")
        want = G.values("hashmin")
    code, steps = ipg.hashmin_noalloc(g.n, _dev(g.row_ptr), _dev(g.col), out)
    assert code == ipg.IP_OK and steps == st.supersteps
    assert np.array_equal(out.cpu().numpy().view(np.uint32), want)
