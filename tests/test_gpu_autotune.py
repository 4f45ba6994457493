"""The autotuner on a 2 x 2 grid of degree-bin cutoffs and a small mode-cutoff
fit (R-MAT scale 12): its output is a loadable JSON of the shape the binding
applies, every cutoff it picks is from the grid, and runs with the tuned cutoffs
give the oracle's results (the cutoffs change only how the work is scheduled)."""
import json

import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2010_08781_gb300 as ipg  # noqa: E402
from paper_2010_08781_gb300 import autotune  # noqa: E402


def test_autotune_small_grid(tmp_path):
    sym = inputs.rmat_graph(12, symmetrize=True, weighted=True, seed=3)
    drc = inputs.rmat_graph(12, seed=3)
    graphs = [("rmat12s", sym), ("rmat12d", drc)]
    bins = autotune.tune_bins(reps=1, graphs=graphs, t1s=(8, 32), t2s=(256, 1024), log=lambda *_: None)
    modes = autotune.tune_modes(specs=[dict(kind="rmat", scale=12, a=0.57, seed=5)], log=lambda *_: None)
    out = tmp_path / "tuned.json"
    out.write_text(json.dumps({"bins": bins, "modes": modes}))
    res = json.loads(out.read_text())
    assert set(res["bins"]) == {"hashmin", "sssp", "pagerank"}
    for app, b in res["bins"].items():
        assert b["t1"] in (8, 32) and b["t2"] in (256, 1024) and len(b["grid_ms"]) == 4
    thr_s, thr_p = res["modes"]["thr_sparse"], res["modes"]["thr_pull"]
    assert 0.0 <= thr_s <= thr_p <= 1.0 and res["modes"]["samples"] > 0
    with ipg.Graph.from_inputs(sym) as G:
        for app in ("hashmin", "sssp"):
            b = res["bins"][app]
            G.run(app, t1=b["t1"], t2=b["t2"], thr_sparse=thr_s, thr_pull=thr_p, policy="threshold")
            want = oracle.run_app(app, sym)[0]
            assert np.array_equal(G.values(app), want), app
    with ipg.Graph.from_inputs(drc) as G:
        b = res["bins"]["pagerank"]
        G.run("pagerank", t1=b["t1"], t2=b["t2"], policy="forced", forced_mode="pull", pr_engine="gather")
        want, _ = oracle.pagerank(drc.n, drc.row_ptr, drc.col, T=30)
        assert float(np.max(np.abs(G.values("pagerank") - want) / want)) <= 1e-5
