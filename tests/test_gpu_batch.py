"""Batched persistent runs against independent oracle runs: every source of a
multi-source SSSP and every instance of a multi-instance Hashmin must match the
oracle bit for bit, with the superstep count each run takes on its own."""
import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2010_08781_gb300 as ipg  # noqa: E402


def _check_sssp(g, sources, dist, st):
    for i, s in enumerate(sources):
        want, ost = oracle.sssp(g.n, g.row_ptr, g.col, g.w, source=int(s))
        assert np.array_equal(dist[i], want), f"source {s}: {int((dist[i] != want).sum())} differ"
        assert st["instance_supersteps"][i] == ost["supersteps"], s
    assert st["halted"] and st["code"] == ipg.IP_OK


@pytest.mark.parametrize("k", [1, 40, 64, 256])
def test_batch_sssp_matches_oracle(k):
    g = inputs.rmat_graph(10 if k == 256 else 12, symmetrize=True, weighted=True, seed=3)
    sources = np.concatenate([[0], inputs.uniform_vertices(g.n, k - 1, seed=k)]).astype(np.uint32)
    with ipg.Graph.from_inputs(g) as G:
        dist, st = G.run_batch_sssp(sources)
    _check_sssp(g, sources, dist, st)


def test_batch_sssp_directed_unweighted_device_output():
    g = inputs.rmat_graph(11, seed=5)  # directed, unweighted (weight 1)
    sources = inputs.uniform_vertices(g.n, 33, seed=9)
    out = torch.empty((33, g.n), dtype=torch.int32, device="cuda")
    with ipg.Graph.from_inputs(g) as G:
        _, st = G.run_batch_sssp(sources, out=out)
        _, st2 = G.run_batch_sssp(sources, out=out)  # the cached graph launch, same results
    _check_sssp(g, sources, out.cpu().numpy().view(np.uint32), st2)
    assert st["supersteps"] == st2["supersteps"]


def test_batch_sssp_duplicate_sources_and_cap():
    g = inputs.path(40, weighted=True)
    sources = np.array([0, 0, 39, 20], np.uint32)
    with ipg.Graph.from_inputs(g) as G:
        dist, st = G.run_batch_sssp(sources)
        _check_sssp(g, sources, dist, st)
        _, st = G.run_batch_sssp(sources, max_supersteps=5)
        assert st["code"] == ipg.IP_E_MAXSTEPS and st["supersteps"] == 5


@pytest.mark.parametrize("engine", ["graph", "persistent"])
def test_batch_hashmin_matches_oracle(engine):
    rng = np.random.default_rng(4)
    gs = [inputs.rmat_sized(int(n), 8, seed=100 + i) for i, n in enumerate(rng.integers(1, 3000, 25))]
    gs.append(inputs.empty_graph(7))
    u, offs = inputs.block_diagonal(gs)
    with ipg.Graph.from_inputs(u) as G:
        labels, st = G.run_batch_hashmin(offs.astype(np.uint32), engine=engine)
    assert st["halted"]
    m = 0
    for i, h in enumerate(gs):
        want, ost = oracle.hashmin(h.n, h.row_ptr, h.col)
        assert np.array_equal(labels[offs[i]:offs[i + 1]], want), i
        assert st["instance_supersteps"][i] == ost["supersteps"], i
        m += int(ost["messages"].sum())
    assert st["supersteps"] == max(st["instance_supersteps"])
    assert st["messages"] == m


def test_batch_errors_and_bounded_barrier_timeout():
    g = inputs.rmat_graph(10, symmetrize=True, weighted=True, seed=2)
    with ipg.Graph.from_inputs(g) as G:
        with pytest.raises(ipg.IPError) as e:
            G.run_batch_sssp(np.zeros(257, np.uint32))
        assert e.value.code == ipg.IP_E_RANGE
        with pytest.raises(ipg.IPError) as e:
            G.run_batch_sssp(np.array([g.n], np.uint32))
        assert e.value.code == ipg.IP_E_RANGE
        with pytest.raises(ipg.IPError) as e:
            G.run_batch_hashmin(np.array([0, 5, 3, g.n], np.uint32))
        assert e.value.code == ipg.IP_E_INVAL
        # a 1 ns bound makes the first barrier wait give up: the kernel exits with an error status
        with pytest.raises(ipg.IPError) as e:
            G.run_batch_sssp(np.array([0, 1], np.uint32), barrier_timeout_ns=1)
        assert e.value.code == ipg.IP_E_TIMEOUT
        # the context is still usable
        dist, st = G.run_batch_sssp(np.array([0, 1], np.uint32))
    _check_sssp(g, [0, 1], dist, st)


def test_batch_full_size_sampled():
    """256 sources on symmetrised R-MAT scale 20, and 1,000 Hashmin instances of
    1k-100k vertices: sampled outputs against the oracle."""
    g = inputs.rmat_graph(20, symmetrize=True, weighted=True, seed=1)
    sources = np.concatenate([[0], inputs.uniform_vertices(g.n, 255, seed=1)]).astype(np.uint32)
    with ipg.Graph.from_inputs(g) as G:
        dist, st = G.run_batch_sssp(sources)
    pick = [0, 1, 128, 255]
    _check_sssp(g, sources[pick], dist[pick], {**st, "instance_supersteps": st["instance_supersteps"][pick]})
    del g, dist
    gs = inputs.hashmin_instances(1000, seed=1)
    u, offs = inputs.block_diagonal(gs)
    with ipg.Graph.from_inputs(u) as G:
        for engine in ("graph", "persistent"):
            labels, st = G.run_batch_hashmin(offs.astype(np.uint32), engine=engine)
            assert st["halted"]
            for i in (0, 1, 499, 998, 999):
                h = gs[i]
                want, ost = oracle.hashmin(h.n, h.row_ptr, h.col)
                assert np.array_equal(labels[offs[i]:offs[i + 1]], want), (engine, i)
                assert st["instance_supersteps"][i] == ost["supersteps"], (engine, i)
