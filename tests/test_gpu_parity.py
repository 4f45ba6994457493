"""GPU parity: the sm_103a library against the CPU oracle, through the C ABI.

Integer apps (Hashmin, SSSP) must match bit for bit, values and per-superstep
frontier counts (active vertices, broadcasters, messages), in every exchange
mode and under random per-superstep mode sequences. FP32 PageRank must be within
max relative error 1e-5 per vertex of the FP64 oracle.
"""
import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # the parity tests need the device; nothing silently falls back
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2010_08781_gb300 as ipg  # noqa: E402

PR_RTOL = 1e-5
MODES = ["push_sparse", "push_dense", "pull"]


def _oracle(app, g, **kw):
    if app == "sssp":
        return oracle.sssp(g.n, g.row_ptr, g.col, g.w, source=kw.get("source", 0))
    if app == "hashmin":
        return oracle.hashmin(g.n, g.row_ptr, g.col)
    return oracle.pagerank(g.n, g.row_ptr, g.col, T=kw.get("T", 30), damping=kw.get("d", 0.85))


def _check_min(G, g, app, ref=None, **opts):
    st = G.run(app, **opts)
    got = G.values(app)
    want, rst = ref if ref is not None else _oracle(app, g, source=opts.get("source", 0))
    assert st.code == ipg.IP_OK and st.halted
    assert np.array_equal(got, want), f"{int((got != want).sum())} values differ"
    assert st.supersteps == rst["supersteps"]
    assert st.active.tolist() == rst["active"].tolist()
    assert st.broadcasters.tolist() == rst["broadcasters"].tolist()
    assert st.messages.tolist() == rst["messages"].tolist()
    return st


def _pr_err(got, want):
    return float(np.max(np.abs(got.astype(np.float64) - want) / np.abs(want)))


# ------------------------------------------------------------------ small graphs
@pytest.fixture(scope="module")
def graphs():
    return {
        "rmat12s": inputs.rmat_graph(12, symmetrize=True, weighted=True, seed=2),
        "rmat11d": inputs.rmat_graph(11, weighted=True, seed=3),
        "er": inputs.er_graph(3000, 9000, seed=4, weighted=True),
        "ragged": inputs.from_edges(1000, *inputs.er_edges(1000, 4000, seed=9), weighted=True),
    }


@pytest.mark.parametrize("app", ["hashmin", "sssp"])
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("name", ["rmat12s", "rmat11d", "er", "ragged"])
def test_min_apps_every_mode(graphs, app, mode, name):
    g = graphs[name]
    with ipg.Graph.from_inputs(g) as G:
        st = _check_min(G, g, app, policy="forced", forced_mode=mode)
        assert all(m == ipg.MODES[mode] for m in st.mode[1:])


@pytest.mark.parametrize("app", ["hashmin", "sssp"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_min_apps_random_mode_sequences(graphs, app, seed):
    g = graphs["rmat12s"]
    rng = np.random.default_rng(seed)
    seq = rng.integers(0, 3, 17).tolist()
    with ipg.Graph.from_inputs(g) as G:
        ref = _oracle(app, g)
        for use_graph in (1, 0):
            st = _check_min(G, g, app, ref=ref, mode_sequence=seq, use_graph=use_graph)
            assert st.mode[1:].tolist() == [seq[(s - 1) % len(seq)] for s in range(1, st.supersteps)]


@pytest.mark.parametrize("app", ["hashmin", "sssp"])
def test_degree_bins_all_paths(graphs, app):
    """Tiny cutoffs put vertices in all three bins (lane, warp, CTA) on a small graph."""
    g = graphs["rmat11d"]
    ref = _oracle(app, g)
    with ipg.Graph.from_inputs(g) as G:
        for t1, t2 in ((1, 2), (2, 8), (4, 64), (64, 100000)):
            for mode in MODES:
                _check_min(G, g, app, ref=ref, policy="forced", forced_mode=mode, t1=t1, t2=t2)


@pytest.mark.parametrize("app", ["hashmin", "sssp"])
def test_threshold_policy_and_host_loop(graphs, app):
    g = graphs["rmat12s"]
    ref = _oracle(app, g)
    with ipg.Graph.from_inputs(g) as G:
        for use_graph in (1, 0):
            st = _check_min(G, g, app, ref=ref, policy="threshold", use_graph=use_graph)
            # the threshold rule is a function of the logged feature f6 = msgs / E
            f6 = st.features[:-1, 6]
            o = ipg.default_options()
            want = np.where(f6 < np.float32(o.thr_sparse), 0, np.where(f6 >= np.float32(o.thr_pull), 2, 1))
            assert st.mode[1:].tolist() == want.tolist()


def test_sssp_other_sources_and_unit_weights(graphs):
    g = graphs["rmat12s"]
    with ipg.Graph.from_inputs(g) as G:
        for s in (1, 77, g.n - 1):
            _check_min(G, g, "sssp", source=s, policy="threshold")
    gu = inputs.rmat_graph(12, symmetrize=True, weighted=False, seed=5)
    with ipg.Graph.from_inputs(gu) as G:
        _check_min(G, gu, "sssp", policy="forced", forced_mode="pull")
        _check_min(G, gu, "sssp", policy="forced", forced_mode="push_sparse")


def test_device_built_csc(graphs):
    g = graphs["rmat11d"]
    with ipg.Graph.from_inputs(g, build_csc_on_device=True) as G:
        for app in ("hashmin", "sssp"):
            _check_min(G, g, app, policy="forced", forced_mode="pull")
        G.run("pagerank", policy="forced", forced_mode="pull")
        want, _ = _oracle("pagerank", g)
        assert _pr_err(G.values("pagerank"), want) <= PR_RTOL


def test_device_pointer_inputs(graphs):
    g = graphs["rmat12s"]
    t = lambda a: torch.from_numpy(a.astype(np.int32)).cuda()  # noqa: E731
    with ipg.Graph(g.n, t(g.row_ptr), t(g.col), t(g.w), symmetric=True) as G:
        _check_min(G, g, "sssp", policy="threshold")
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        G.values(out=out)
        want, _ = _oracle("sssp", g)
        assert np.array_equal(out.cpu().numpy().view(np.uint32), want)


# ------------------------------------------------------------------ edge cases
def test_edge_cases():
    cases = [inputs.empty_graph(1), inputs.empty_graph(37), inputs.path(33), inputs.star(70),
             inputs.from_edges(3, [0, 1, 1, 2], [0, 1, 2, 2]),  # self-loops
             inputs.directed_cycle(65), inputs.complete_digraph(40)]
    for g in cases:
        with ipg.Graph.from_inputs(g) as G:
            for app in ("hashmin", "sssp"):
                for mode in MODES:
                    _check_min(G, g, app, policy="forced", forced_mode=mode)
            for mode in ("pull", "push_dense"):
                G.run("pagerank", policy="forced", forced_mode=mode)
                want, _ = _oracle("pagerank", g)
                assert _pr_err(G.values("pagerank"), want) <= PR_RTOL


def test_superstep_cap_and_errors(graphs):
    g = inputs.path(50)
    with ipg.Graph.from_inputs(g, selector=None) as G:
        st = G.run("hashmin", max_supersteps=5)
        assert st.code == ipg.IP_E_MAXSTEPS and st.supersteps == 5 and not st.halted
        ref, _ = oracle.hashmin(g.n, g.row_ptr, g.col, max_supersteps=5)
        assert np.array_equal(G.values("hashmin"), ref)
        with pytest.raises(ipg.IPError) as e:
            G.run("sssp", source=g.n)
        assert e.value.code == ipg.IP_E_RANGE
        with pytest.raises(ipg.IPError):
            G.run("hashmin", policy="mlp")  # no selector loaded
        with pytest.raises(ipg.IPError):
            G.run("hashmin", t1=10, t2=5)
    with pytest.raises(ipg.IPError) as e:
        ipg.Graph(4, np.array([0, 1, 2, 3, 4]), np.array([1, 2, 3, 9]))
    assert e.value.code == ipg.IP_E_RANGE
    with pytest.raises(ipg.IPError) as e:
        ipg.Graph(4, np.array([0, 2, 1, 3, 4]), np.array([1, 2, 3, 0]))
    assert e.value.code == ipg.IP_E_INVAL
    bad = torch.tensor([0, 1, 2, 3, 4], dtype=torch.int32, device="cuda")
    with pytest.raises(ipg.IPError) as e:
        ipg.Graph(4, bad, torch.tensor([1, 2, 3, 9], dtype=torch.int32, device="cuda"))
    assert e.value.code == ipg.IP_E_RANGE


# ------------------------------------------------------------------ PageRank
@pytest.fixture(scope="module")
def rmat16():
    # scale 16, edge factor 16, (.57,.19,.19,.05), seed 1, duplicates removed
    return inputs.rmat_graph(16, seed=1)


@pytest.fixture(scope="module")
def pr16_ref(rmat16):
    return _oracle("pagerank", rmat16)


@pytest.mark.parametrize("mode", ["pull", "push_dense"])
def test_pagerank_scale16_parity(rmat16, pr16_ref, mode):
    with ipg.Graph.from_inputs(rmat16) as G:
        st = G.run("pagerank", policy="forced", forced_mode=mode)
        got = G.values("pagerank")
    want, rst = pr16_ref
    assert st.supersteps == rst["supersteps"] == 31
    assert st.active.tolist() == rst["active"].tolist()
    assert st.broadcasters.tolist() == rst["broadcasters"].tolist()
    assert st.messages.tolist() == rst["messages"].tolist()
    assert _pr_err(got, want) <= PR_RTOL


def test_pagerank_bins_and_closed_forms(rmat16, pr16_ref):
    want, _ = pr16_ref
    with ipg.Graph.from_inputs(rmat16) as G:
        for t1, t2 in ((1, 2), (4, 64), (256, 100000)):
            G.run("pagerank", policy="forced", forced_mode="pull", t1=t1, t2=t2)
            assert _pr_err(G.values("pagerank"), want) <= PR_RTOL
    k = 300
    d = 0.85
    N = k + 1
    rc = (1 + d * k) / (N * (1 + d))
    rl = (1 - d) / N + d * rc / k
    ec, el = 1.0 / N - rc, 1.0 / N - rl
    for _ in range(30):
        ec, el = d * k * el, d * ec / k
    with ipg.Graph.from_inputs(inputs.star(k)) as G:
        G.run("pagerank", t2=64)  # the centre goes through the CTA path
        r = G.values("pagerank").astype(np.float64)
    assert abs(r[0] - (rc + ec)) / (rc + ec) <= PR_RTOL
    assert np.max(np.abs(r[1:] - (rl + el)) / (rl + el)) <= PR_RTOL


# ------------------------------------------------------------------ full size
@pytest.fixture(scope="module")
def rmat22s():
    # symmetrised R-MAT scale 22, edge factor 16, weights uniform in [1, 255], seed 1
    return inputs.rmat_graph(22, symmetrize=True, weighted=True, seed=1)


@pytest.mark.parametrize("app", ["hashmin", "sssp"])
def test_full_size_scale22(rmat22s, app):
    g = rmat22s
    ref = _oracle(app, g)
    with ipg.Graph.from_inputs(g) as G:
        _check_min(G, g, app, ref=ref, policy="threshold")
        _check_min(G, g, app, ref=ref, policy="forced", forced_mode="pull")


@pytest.mark.parametrize("app", ["hashmin", "sssp", "pagerank"])
def test_label_collection_and_kernel_profiling_keep_values(graphs, app):
    """Timing every mode per superstep (selector training labels) or every kernel
    leaves the values and the per-superstep counts unchanged."""
    g = graphs["rmat12s"]
    with ipg.Graph.from_inputs(g) as G:
        if app == "pagerank":
            want, _ = _oracle("pagerank", g)
            for kw in (dict(collect_labels=1), dict(profile_kernels=1)):
                st = G.run("pagerank", **kw)
                assert _pr_err(G.values("pagerank"), want) <= PR_RTOL
            return
        ref = _oracle(app, g)
        st = _check_min(G, g, app, ref=ref, policy="threshold", collect_labels=1)
        assert (st.mode_ms[1:] > 0).all()
        st = _check_min(G, g, app, ref=ref, policy="threshold", profile_kernels=1)
        assert (st.kernel_ms[1:, 1] > 0).all() and (st.kernel_ms[1:, 2] > 0).all()
