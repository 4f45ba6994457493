"""Autotuner for the scheduling cutoffs of the superstep engine.

Degree-bin cutoffs: t1 (largest degree handled by one lane) and t2 (smallest
degree handled by whole CTAs in 4096-edge chunks) are chosen per app by a grid
search of whole runs (device time, median of repeats) on seeded R-MAT graphs.
Mode cutoffs: the threshold rule's two cutoffs on messages/E are fitted to
per-superstep timings of all three exchange modes (the selector's label logs).

Both cutoff sets are tuned twice: on graphs renumbered by degree class (the
binding's default from 2^20 edges) and in the caller's order; the binding picks the
set that matches the graph.

Command line (on a GPU machine):
    python -m paper_2010_08781_gb300.autotune --out FILE
The result is written as JSON; the package applies paper_2010_08781_gb300/tuned_defaults.json
(if present) as the defaults of its run options.
"""
from __future__ import annotations

import argparse
import json
import statistics
import time

import numpy as np

from . import Graph

T1S = (8, 16, 32, 64, 128)
T2S = (256, 512, 1024, 2048, 4096)


def _graphs():
    import inputs
    yield "rmat20s", inputs.rmat_graph(20, symmetrize=True, weighted=True, seed=3)
    yield "rmat22s", inputs.rmat_graph(22, symmetrize=True, weighted=True, seed=3)
    yield "rmat22d", inputs.rmat_graph(22, seed=3)


def time_run(G, app, reps, **kw):
    ts = [G.run(app, **kw).elapsed_ms for _ in range(reps)]
    return statistics.median(ts)


def tune_bins(reps=3, relabel=True, log=print, graphs=None, t1s=T1S, t2s=T2S):
    """Grid search of (t1, t2) per app; total time over the tuning graphs (name,
    inputs.Graph pairs; a name ending in "d" marks a directed graph, tuned for
    PageRank), stored renumbered by degree class (relabel=True) or in the caller's
    order."""
    totals = {app: {} for app in ("hashmin", "sssp", "pagerank")}
    for name, g in (graphs if graphs is not None else _graphs()):
        with Graph.from_inputs(g, relabel=relabel) as G:
            apps = ("pagerank",) if name.endswith("d") else ("hashmin", "sssp")
            for app in apps:
                # the degree bins schedule the CSC gather engine (the blocked engine has its own layout)
                kw = dict(policy="forced", forced_mode="pull", pr_engine="gather") if app == "pagerank" else {}
                for t1 in t1s:
                    for t2 in t2s:
                        G.run(app, t1=t1, t2=t2, **kw)  # warm-up (bins rebuilt for the new cutoffs)
                        ms = time_run(G, app, reps, t1=t1, t2=t2, **kw)
                        totals[app][(t1, t2)] = totals[app].get((t1, t2), 0.0) + ms
            log(f"tuned bins on {name}")
    best = {}
    for app, d in totals.items():
        if not d:
            continue
        (t1, t2), ms = min(d.items(), key=lambda kv: kv[1])
        best[app] = {"t1": t1, "t2": t2, "ms": round(ms, 4),
                     "grid_ms": {f"{a},{b}": round(v, 4) for (a, b), v in sorted(d.items())}}
    return best


def tune_modes(log=print, specs=None):
    from . import selector
    if specs is None:
        specs = [dict(kind="rmat", scale=s, a=a, seed=5) for s in (20, 22) for a in (0.45, 0.57, 0.65)]
    X, T, _ = selector.collect_many(specs, log=log)
    a, b = selector.tune_threshold(X, T)
    return {"thr_sparse": a, "thr_pull": b, "samples": int(X.shape[0])}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    t0 = time.time()
    bins = tune_bins(args.reps)
    bins_caller = tune_bins(args.reps, relabel=False)
    modes = tune_modes()
    res = {"bins": bins, "bins_caller_order": bins_caller, "modes": modes, "seconds": round(time.time() - t0, 1),
           "graphs": "R-MAT scale 20/22 symmetrised weighted (seed 3) for Hashmin/SSSP, directed scale 22 for PageRank; "
                     "mode cutoffs from per-mode superstep timings on R-MAT scale 20/22, a in {.45,.57,.65}, seed 5"}
    with open(args.out, "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps({k: ({a: {kk: vv for kk, vv in v.items() if kk != "grid_ms"} for a, v in res[k].items()}
                          if k.startswith("bins") else v) for k, v in res.items()}))


if __name__ == "__main__":
    main()
