"""Learned push/pull mode selector: log collection, training, evaluation.

The superstep engine logs, for every superstep s, the 8 frontier features
computed after superstep s-1 (the selector's input) and — with
``collect_labels=1`` — the measured time of each of the three exchange modes
delivering into s, all started from the same state. A training sample is
(features, fastest mode), weighted by the time at stake (slowest - fastest).

Training runs on the GPU through the library's own kernels (ip_mlp_backward,
ip_mlp_adam); this module only moves tensors and loops. The trained network is
packed by ip_mlp_pack into the blob that ip_set_selector loads.

Command line (on a GPU machine):
    python -m paper_2010_08781_gb300.selector train --out DIR
writes DIR/selector_weights.bin, DIR/selector_report.json and the logs;
    python -m paper_2010_08781_gb300.selector evaluate --out DIR
times whole runs of the shipped selector against the threshold rule on the
held-out graphs of held_out_graphs() (DIR/selector_held_out.json).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import time

import numpy as np

from . import (MLP_PARAMS, N_FEATURES, SELECTOR_BYTES, Graph, IPError, _check, load)

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "selector_weights.bin")
FEATURES = ("log1p broadcasters", "log1p messages (out-edges of broadcasters)", "log1p mean out-degree",
            "log1p max out-degree", "broadcasters / V", "log1p last superstep time [ns]", "messages / E",
            "log frontier growth")
MODE_NAMES = ("push_sparse", "push_dense", "pull")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


# ----------------------------------------------------------------- logs
def collect(G: Graph, app: str, source: int = 0, policy: str = "threshold"):
    """Per-superstep (features, per-mode ms) of one run; the trajectory does not
    depend on the policy."""
    kw = dict(source=source) if app == "sssp" else {}
    st = G.run(app, policy=policy, collect_labels=1, **kw)
    X = st.features[: st.supersteps - 1].astype(np.float32)
    T = st.mode_ms[1: st.supersteps].astype(np.float32)
    return X, T


def labels_of(T):
    """Fastest mode and the time at stake (ms) per sample."""
    y = T.argmin(axis=1).astype(np.int32)
    w = (T.max(axis=1) - T.min(axis=1)).astype(np.float32) + np.float32(1e-3)
    return y, w


def threshold_modes(X, thr_sparse=0.02, thr_pull=0.15):
    """The fixed rule of the engine on feature 6 (messages / E), in FP32 like the kernel."""
    f6 = X[:, 6].astype(np.float32)
    return np.where(f6 < np.float32(thr_sparse), 0, np.where(f6 >= np.float32(thr_pull), 2, 1)).astype(np.int32)


def total_time(modes, T):
    return float(T[np.arange(T.shape[0]), modes].sum())


# ----------------------------------------------------------------- training on the GPU
class Trainer:
    """FP32 master parameters on the device, trained by the library's kernels."""

    def __init__(self, mu, sd, seed=0):
        import torch
        self.torch = torch
        L = load()
        rng = np.random.default_rng(seed)
        p = np.zeros(MLP_PARAMS, np.float32)
        o = 0
        for fan_in, fan_out in ((8, 32), (32, 32), (32, 3)):
            p[o:o + fan_in * fan_out] = rng.normal(0, np.sqrt(2.0 / fan_in), fan_in * fan_out)
            o += fan_in * fan_out + fan_out  # biases stay 0
        dev = torch.device("cuda")
        self.p = torch.from_numpy(p).to(dev)
        self.musd = torch.from_numpy(np.concatenate([mu, sd]).astype(np.float32)).to(dev)
        self.m = torch.zeros_like(self.p)
        self.v = torch.zeros_like(self.p)
        self.g = torch.zeros_like(self.p)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self.ws_bytes = L.ip_mlp_workspace_bytes()
        self.ws = torch.empty(self.ws_bytes // 4 + 1, dtype=torch.float32, device=dev)
        self.t = 0
        self.L = L

    def _dev(self, a, dtype):
        return self.torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()

    def logits(self, X):
        Xd = self._dev(X, np.float32)
        out = self.torch.empty((X.shape[0], 3), dtype=self.torch.float32, device="cuda")
        _check(self.L.ip_mlp_forward(_ptr(self.p), _ptr(self.musd), _ptr(Xd), X.shape[0], _ptr(out), None),
               "ip_mlp_forward")
        return out.cpu().numpy()

    def gradient(self, Xd, yd, wd, n, wtot):
        _check(self.L.ip_mlp_backward(_ptr(self.p), _ptr(self.musd), _ptr(Xd), _ptr(yd), _ptr(wd), n,
                                      ctypes.c_float(wtot), _ptr(self.g), _ptr(self.loss), _ptr(self.ws),
                                      self.ws_bytes, None), "ip_mlp_backward")
        return self.g, self.loss

    def fit(self, X, y, w, steps=3000, lr=3e-3):
        Xd, yd, wd = self._dev(X, np.float32), self._dev(y, np.int32), self._dev(w, np.float32)
        wtot = float(w.sum())
        hist = []
        for _ in range(steps):
            self.gradient(Xd, yd, wd, X.shape[0], wtot)
            self.t += 1
            _check(self.L.ip_mlp_adam(_ptr(self.p), _ptr(self.g), _ptr(self.m), _ptr(self.v), MLP_PARAMS,
                                      ctypes.c_float(lr), ctypes.c_float(0.9), ctypes.c_float(0.999),
                                      ctypes.c_float(1e-8), self.t, None), "ip_mlp_adam")
            if self.t % 250 == 0:
                hist.append(float(self.loss.item()))
        return hist

    def blob(self) -> bytes:
        out = self.torch.zeros(SELECTOR_BYTES, dtype=self.torch.uint8, device="cuda")
        _check(self.L.ip_mlp_pack(_ptr(self.p), _ptr(self.musd), _ptr(out), None), "ip_mlp_pack")
        return bytes(out.cpu().numpy().tobytes())


def normalisation(X, masked=()):
    """Per-feature mean and spread; a masked feature gets mean 0 and spread 1e30, so
    its normalised input is ~0 in training and in the engine alike (the network
    ignores it without a change of the blob layout)."""
    mu = X.mean(axis=0).astype(np.float32)
    sd = (X.std(axis=0) + 1e-3).astype(np.float32)
    for i in masked:
        mu[i], sd[i] = 0.0, 1e30
    return mu, sd


def load_default_blob():
    if os.path.exists(DEFAULT_WEIGHTS):
        with open(DEFAULT_WEIGHTS, "rb") as f:
            b = f.read()
        if len(b) == SELECTOR_BYTES:
            return b
    return None


# ----------------------------------------------------------------- workloads
def training_graphs():
    """R-MAT scales 18-24 with varied (a, b, c), d = .05, plus Erdos-Renyi graphs;
    symmetrised, weights in [1, 255]."""
    specs = []
    for scale in (18, 20, 22):
        for a in (0.45, 0.57, 0.65):
            for seed in (1, 2, 3):
                specs.append(dict(kind="rmat", scale=scale, a=a, seed=seed))
        for seed in (1, 2):
            specs.append(dict(kind="er", scale=scale, a=None, seed=seed))
    for a in (0.45, 0.57, 0.65):
        specs.append(dict(kind="rmat", scale=24, a=a, seed=1))
    specs.append(dict(kind="er", scale=24, a=None, seed=1))
    return specs


def evaluation_graphs():
    """Held out (seeds never used in training): R-MAT scale 24 with a = .57."""
    return [dict(kind="rmat", scale=24, a=0.57, seed=s) for s in (11, 12, 13)]


def tune_threshold(X, T):
    """Grid search of the threshold rule's two cutoffs on logged supersteps
    (minimum total time of the chosen modes)."""
    grid = np.unique(np.concatenate([[0.0], np.logspace(-5, 0, 101)]).astype(np.float32))
    best = None
    for i, a in enumerate(grid):
        for b in grid[i:]:
            t = total_time(threshold_modes(X, a, b), T)
            if best is None or t < best[0]:
                best = (t, float(a), float(b))
    return best[1], best[2]


def make_graph(spec):
    import inputs
    if spec["kind"] == "er":
        n = 1 << spec["scale"]
        return inputs.er_graph(n, 8 * n, seed=spec["seed"], symmetrize=True, weighted=True)
    a = spec["a"]
    b = c = (1.0 - a - 0.05) / 2
    return inputs.rmat_graph(spec["scale"], 16, a, b, c, seed=spec["seed"], symmetrize=True, weighted=True,
                             permute_seed=spec.get("permute"))


def collect_many(specs, sssp_sources=4, log=print):
    import inputs
    Xs, Ts, meta = [], [], []
    for spec in specs:
        t0 = time.time()
        g = make_graph(spec)
        with Graph.from_inputs(g) as G:
            runs = [("hashmin", 0)] + [("sssp", int(s)) for s in
                                       [0] + inputs.uniform_vertices(g.n, sssp_sources - 1, seed=spec["seed"] + 7).tolist()]
            for app, src in runs:
                X, T = collect(G, app, src)
                Xs.append(X)
                Ts.append(T)
                meta += [dict(spec, app=app, source=src, superstep=i + 1) for i in range(X.shape[0])]
        log(f"collected {spec} in {time.time() - t0:.1f}s")
        del g
    return np.concatenate(Xs), np.concatenate(Ts), meta


def report(name, X, T, modes_by_policy):
    out = {"samples": int(X.shape[0]), "best_ms": round(float(T.min(axis=1).sum()), 4)}
    for pol, modes in modes_by_policy.items():
        out[pol + "_ms"] = round(total_time(modes, T), 4)
    for m in range(3):
        out["forced_" + MODE_NAMES[m] + "_ms"] = round(float(T[:, m].sum()), 4)
    return out


def live_compare(specs, blob, thr_sparse, thr_pull, reps=5):
    """Whole runs in the device-driven loop: median ms per policy, per app."""
    out = []
    for spec in specs:
        g = make_graph(spec)
        with Graph.from_inputs(g, selector=blob) as G:
            for app in ("hashmin", "sssp"):
                row = dict(spec, app=app)
                for name, kw in (("mlp", dict(policy="mlp")),
                                 ("threshold_tuned", dict(policy="threshold", thr_sparse=thr_sparse,
                                                          thr_pull=thr_pull)),
                                 ("pull", dict(policy="forced", forced_mode="pull"))):
                    ts = sorted(G.run(app, **kw).elapsed_ms for _ in range(reps))
                    row[name + "_ms"] = round(ts[len(ts) // 2], 4)
                out.append(row)
    return out


def held_out_graphs():
    """A wider held-out set than evaluation_graphs (no seed of any training graph,
    several shapes): R-MAT 22 like the benchmark's secondary line but other seeds,
    R-MAT 23 with a = .45 and .65, R-MAT 24 (a = .57), Erdos-Renyi at 2^22 and 2^24
    vertices, and a randomly permuted R-MAT 22."""
    specs = [dict(kind="rmat", scale=22, a=0.57, seed=s) for s in (11, 12)]
    specs += [dict(kind="rmat", scale=23, a=a, seed=11) for a in (0.45, 0.65)]
    specs += [dict(kind="rmat", scale=24, a=0.57, seed=s) for s in (11, 12)]
    specs += [dict(kind="er", scale=22, a=None, seed=11), dict(kind="er", scale=24, a=None, seed=11)]
    specs += [dict(kind="rmat", scale=22, a=0.57, seed=13, permute=17)]
    return specs


def evaluate_live(specs, reps=7, sources=3, log=print):
    """Whole runs of both apps in the device-driven loop, learned selector against
    the threshold rule (the engine's defaults): the two policies alternate run by
    run (so drift hits both alike); median ms per (graph, app, source)."""
    import inputs
    rows = []
    for spec in specs:
        g = make_graph(spec)
        with Graph.from_inputs(g) as G:
            runs = [("hashmin", 0)] + [("sssp", int(x)) for x in
                                       [0] + inputs.uniform_vertices(g.n, sources - 1, seed=spec["seed"] + 29).tolist()]
            for app, src in runs:
                kw = dict(source=src) if app == "sssp" else {}
                ts = {"mlp": [], "threshold": []}
                for _ in range(reps):
                    for pol in ("mlp", "threshold"):
                        ts[pol].append(G.run(app, policy=pol, **kw).elapsed_ms)
                row = dict(spec, app=app, source=src, edges=g.m,
                           mlp_ms=round(float(np.median(ts["mlp"])), 4),
                           threshold_ms=round(float(np.median(ts["threshold"])), 4))
                row["gain"] = round(row["threshold_ms"] / row["mlp_ms"] - 1.0, 4)
                rows.append(row)
                log(json.dumps(row))
        del g
    summary = {}
    for app in ("hashmin", "sssp"):
        r = [x for x in rows if x["app"] == app]
        tot_m, tot_t = sum(x["mlp_ms"] for x in r), sum(x["threshold_ms"] for x in r)
        summary[app] = {"runs": len(r), "mlp_ms": round(tot_m, 3), "threshold_ms": round(tot_t, 3),
                        "gain_total_time": round(tot_t / tot_m - 1.0, 4),
                        "gain_geomean": round(float(np.exp(np.mean([np.log(1 + x["gain"]) for x in r]))) - 1.0, 4),
                        "runs_won": int(sum(x["gain"] > 0 for x in r))}
    return rows, summary


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train", "evaluate"])
    ap.add_argument("--out", default=".")
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--mask", type=int, nargs="*", default=[],
                    help="feature indices the network ignores (e.g. 5: the last superstep's time)")
    args = ap.parse_args()
    os.makedirs(args.out, exist_ok=True)
    if args.cmd == "evaluate":
        rows, summary = evaluate_live(held_out_graphs())
        with open(os.path.join(args.out, "selector_held_out.json"), "w") as f:
            json.dump({"graphs": held_out_graphs(), "runs": rows, "summary": summary}, f, indent=1)
        print(json.dumps(summary))
        return
    Xtr, Ttr, meta_tr = collect_many(training_graphs())
    Xev, Tev, meta_ev = collect_many(evaluation_graphs())
    np.savez_compressed(os.path.join(args.out, "selector_logs.npz"), Xtr=Xtr, Ttr=Ttr, Xev=Xev, Tev=Tev)
    y, w = labels_of(Ttr)
    thr_sparse, thr_pull = tune_threshold(Xtr, Ttr)
    mu, sd = normalisation(Xtr, args.mask)
    tr = Trainer(mu, sd)
    t0 = time.time()
    hist = tr.fit(Xtr, y, w, steps=args.steps, lr=args.lr)
    train_s = time.time() - t0
    blob = tr.blob()
    with open(os.path.join(args.out, "selector_weights.bin"), "wb") as f:
        f.write(blob)
    pred_tr = tr.logits(Xtr).argmax(axis=1)
    pred_ev = tr.logits(Xev).argmax(axis=1)
    rep = {
        "network": "8-32-32-3 MLP, BF16 weights, FP32 accumulation",
        "features": FEATURES,
        "masked_features": [FEATURES[i] for i in args.mask],
        "training_graphs": training_graphs(),
        "evaluation_graphs": evaluation_graphs(),
        "train_steps": args.steps, "lr": args.lr, "train_seconds": round(train_s, 2), "loss_history": hist,
        "tuned_threshold": {"thr_sparse": thr_sparse, "thr_pull": thr_pull},
        "train": report("train", Xtr, Ttr, {"mlp": pred_tr, "threshold_default": threshold_modes(Xtr),
                                            "threshold_tuned": threshold_modes(Xtr, thr_sparse, thr_pull)}),
        "train_accuracy": float((pred_tr == y).mean()),
        "eval": report("eval", Xev, Tev, {"mlp": pred_ev, "threshold_default": threshold_modes(Xev),
                                          "threshold_tuned": threshold_modes(Xev, thr_sparse, thr_pull)}),
        "eval_accuracy": float((pred_ev == labels_of(Tev)[0]).mean()),
    }
    rep["live_eval"] = live_compare(evaluation_graphs(), blob, thr_sparse, thr_pull)
    with open(os.path.join(args.out, "selector_report.json"), "w") as f:
        json.dump(rep, f, indent=1)
    print(json.dumps({k: rep[k] for k in ("tuned_threshold", "train", "eval", "train_accuracy", "eval_accuracy",
                                          "train_seconds", "live_eval")}))


if __name__ == "__main__":
    main()
