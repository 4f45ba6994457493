#!/usr/bin/env python3
"""Benchmark of the synchronous vertex-centric superstep library on one GB300.

Workload (one "step"): Hashmin connected components and SSSP from vertex 0 on
the symmetrised R-MAT graph of scale 22 (4,194,304 vertices, edge factor 16,
(a,b,c,d) = (.57,.19,.19,.05), seed 1, duplicates removed, uint32 weights
uniform in [1, 255]), each run to global halt with the default mode policy.

Metric: GTEPS = messages sent (sum over supersteps of the out-degrees of the
broadcasting vertices, both apps) / step time. The JSON line also carries the
roofline of the dominant kernel (algorithmic bytes / CUDA-event time against
the measured HBM copy bandwidth), the end-to-end number through the C ABI with
host buffers, and the CPU oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

SCALE = 22
EDGE_FACTOR = 16
METRIC = "GTEPS & % HBM BW per app (PageRank/Hashmin/SSSP); learned vs fixed push/pull"
WORKLOAD = ("Hashmin + SSSP(source 0) on symmetrised R-MAT scale 22, edge factor 16, "
            "(a,b,c,d)=(.57,.19,.19,.05), seed 1, duplicates removed, uint32 weights in [1,255]")
L2_BYTES = 129 * 1024 * 1024


def build_graph(scale=SCALE):
    import inputs
    return inputs.rmat_graph(scale, edge_factor=EDGE_FACTOR, a=0.57, b=0.19, c=0.19, seed=1, symmetrize=True,
                             weighted=True, wseed=1)


def measured_traffic(kernel):
    """DRAM bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum) of a
    kernel on the workload it is reported for, from profiles/traffic.json (written
    from an ncu capture of the same command; None when not captured)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel)
    return None if e is None else e.get("bytes_per_launch")


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons every INTERVAL_MS, started
    before the warm-up; summary() keeps the samples whose timestamps fall inside the
    marked timed region (or the nearest one when the region is shorter than the
    sampling interval)."""
    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 50

    def __init__(self, device_index):
        import tempfile
        self.idx = device_index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix=f"ipregel_clocks{device_index}_", suffix=".csv")
        os.close(fd)
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return self
        deadline = time.time() + 5.0  # wait for the first sample
        while time.time() < deadline and self.proc.poll() is None and os.path.getsize(self.path) == 0:
            time.sleep(0.02)
        return self

    def start(self):
        self.t0 = time.time()

    def stop(self):
        self.t1 = time.time()

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(2 * self.INTERVAL_MS / 1e3)  # a sample after the region
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def _rows(self):
        from datetime import datetime
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 10:
                continue
            try:
                t = datetime.strptime(p[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((t, float(p[2]), float(p[3]), p))
            except ValueError:
                continue
        return rows

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = self._rows()
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        window = "timed region"
        sel = rows
        if self.t0 is not None and self.t1 is not None:
            sel = [r for r in rows if self.t0 <= r[0] <= self.t1]
            if not sel:  # region shorter than the interval: the first sample after its start
                after = [r for r in rows if r[0] >= self.t0]
                sel = after[:1] or rows[-1:]
                window = "nearest sample after the start of the timed region"
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, _, _, p in sel:
            for n, v in zip(names, p[6:10]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(r[1] for r in sel), "sm_max_mhz": max(r[2] for r in sel),
                "reasons": sorted(reasons), "samples": len(sel), "window": window,
                "power_w_median": statistics.median(float(r[3][4]) for r in sel) if sel else None}


# ----------------------------------------------------------------- kernel byte models
def launches_of(mode_seq, app):
    """Kernels one run launches: init + selector, then per superstep the mode's kernels + selector."""
    n = 2
    for m in mode_seq[1:]:
        if app == "pagerank":
            n += 2 if m == 2 else 3
        else:
            n += 4 if m == 0 else 3
    return n


def exchange_bytes(app, mode, V, E, msgs_prev, bcast_prev, recipients):
    """Algorithmic bytes of one exchange launch delivering the broadcasts of the previous superstep.

    pull:        4(V+1) offsets + 4E in-edge sources + V/8 broadcast bitmap + 4 per gathered
                 broadcast value (msgs_prev) [+ 4 per gathered weight, SSSP] + 4 per recipient mailbox
    push:        per sender 8 (offsets) + 4 (value) [+ 4 queue entry, sparse]; per message 4 (target)
                 [+ 4 weight, SSSP] + 4 (mailbox combine); bitmap V/8 (dense)
    PageRank pull (fused with apply): 4(V+1) + 4E + 4E gathers + 16V (inv out-degree, rank, next value)."""
    w = 4 if app == "sssp" else 0
    if app == "pagerank":
        if mode == 2:
            return 4 * (V + 1) + 8 * E + 16 * V
        return 4 * (V + 1) + 8 * E + 4 * V  # push: offsets, targets, atomic adds, values
    if mode == 2:
        return 4 * (V + 1) + 4 * E + V / 8 + (4 + w) * msgs_prev + 4 * recipients
    per_sender = 12 + (4 if mode == 0 else 0)
    return per_sender * bcast_prev + (8 + w) * msgs_prev + (V / 8 if mode == 1 else 0)


KERNEL_NAMES = {("pull", "hashmin"): "k_pull<Hashmin>", ("pull", "sssp"): "k_pull<SSSP>",
                ("push_dense", "hashmin"): "k_push<Hashmin,dense>", ("push_dense", "sssp"): "k_push<SSSP,dense>",
                ("push_sparse", "hashmin"): "k_push<Hashmin,sparse>",
                ("push_sparse", "sssp"): "k_push<SSSP,sparse>", ("pull", "pagerank"): "k_pr_pull"}
MODE_NAMES = {0: "push_sparse", 1: "push_dense", 2: "pull"}


# ----------------------------------------------------------------- replicas
def reduce_over_ranks(total_ms, msgs, world, device=None):
    """Whole-job figures of independent replicas: the slowest rank's time and the
    messages of all ranks (no data-path collective; two scalars per run)."""
    if world <= 1:
        return float(total_ms), float(msgs)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_ms), float(msgs)], dtype=torch.float64, device=device)
    tmax, tsum = t.clone(), t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax[0].item()), float(tsum[1].item())


# ----------------------------------------------------------------- GPU arm
def run_gpu(args, rank, world, local_rank):
    import torch
    import paper_2010_08781_gb300 as ipg

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    g = build_graph(args.scale)
    V, E = g.n, g.m
    # pinned host copies of the inputs (for the end-to-end leg)
    pin = {k: torch.from_numpy(getattr(g, k).view(np.int32)).pin_memory() for k in ("row_ptr", "col", "w")}
    with torch.cuda.stream(stream):
        G = ipg.Graph(V, pin["row_ptr"], pin["col"], pin["w"], symmetric=True, stream=stream)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    opts = dict(policy=args.policy, stream=stream)

    def step():
        a = G.run("hashmin", **opts)
        b = G.run("sssp", source=0, **opts)
        return a, b

    clk = ClockSampler(local_rank).__enter__()  # sampling from before the warm-up
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    msgs = 0
    launches = 0
    per_app = {"hashmin": [], "sssp": []}
    clk.start()
    try:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()  # evict the previous step's working set from L2 (outside the timed events)
                ev[i][0].record(stream)
            a, b = step()
            with torch.cuda.stream(stream):
                ev[i][1].record(stream)
            msgs += int(a.messages.sum()) + int(b.messages.sum())
            launches += launches_of(a.mode.tolist(), "hashmin") + launches_of(b.mode.tolist(), "sssp")
            per_app["hashmin"].append(a)
            per_app["sssp"].append(b)
        torch.cuda.synchronize()
    finally:
        clk.stop()
        clk.__exit__(None, None, None)
    step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    total_ms, msgs_all = reduce_over_ranks(sum(step_ms), msgs, world, dev)
    value = msgs_all / (total_ms * 1e-3) / 1e9

    # ---------------------------------------------------------- roofline of the dominant kernel
    peak, peak_kind = measured_peaks()
    kern = {}  # name -> [total ms, total bytes, launches]
    # the timed runs' own mode sequences are replayed (the learned selector reads the
    # last superstep's time, which events and profilers change)
    seqs = {app: per_app[app][-1].mode[1:per_app[app][-1].supersteps].tolist() for app in ("hashmin", "sssp")}
    for _ in range(args.steps):
        for app in ("hashmin", "sssp"):
            st = G.run(app, profile_kernels=1, stream=stream, mode_sequence=seqs[app])
            for s in range(1, st.supersteps):
                mode = int(st.mode[s])
                name = KERNEL_NAMES[(MODE_NAMES[mode], app)]
                by = exchange_bytes(app, mode, V, E, int(st.messages[s - 1]), int(st.broadcasters[s - 1]),
                                    int(st.active[s]))
                k = kern.setdefault(name, [0.0, 0.0, 0])
                k[0] += float(st.kernel_ms[s, 1])
                k[1] += by
                k[2] += 1
                a = kern.setdefault("k_apply_" + ("queue" if mode == 0 else "bitmap"), [0.0, 0.0, 0])
                a[0] += float(st.kernel_ms[s, 2])
                a[2] += 1
    dom = max((n for n in kern if kern[n][1] > 0), key=lambda n: kern[n][0])
    d_ms, d_bytes, d_n = kern[dom]
    achieved = d_bytes / (d_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": measured_traffic(dom), "launches_per_step": d_n / args.steps,
                "avg_launch_us": round(1e3 * d_ms / d_n, 2)}
    total_k = sum(v[0] for v in kern.values())
    roofline["share_of_kernel_time"] = round(d_ms / total_k, 3)

    # ---------------------------------------------------------- end to end through the C ABI, host buffers
    e2e_ms = []
    h2d = 4 * (V + 1) + 8 * E  # offsets, targets, weights
    d2h = 2 * 4 * V
    out = torch.empty(V, dtype=torch.int32).pin_memory()
    for i in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with ipg.Graph(V, pin["row_ptr"], pin["col"], pin["w"], symmetric=True, stream=stream) as H:
            H.run("hashmin", **opts)
            H.values(out=out, stream=stream)
            H.run("sssp", source=0, **opts)
            H.values(out=out, stream=stream)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_value = (msgs / args.steps) / (statistics.median(e2e_ms) * 1e-3) / 1e9

    # ---------------------------------------------------------- per-app and per-policy detail
    detail = {}
    for app in ("hashmin", "sssp"):
        runs = per_app[app]
        ms = statistics.median(r.elapsed_ms for r in runs)
        m = int(runs[0].messages.sum())
        detail[app] = {"gteps": round(m / (ms * 1e-3) / 1e9, 2), "ms": round(ms, 4), "supersteps": runs[0].supersteps,
                       "messages": m, "modes": runs[0].mode[1:].tolist()}
        pol = {}
        for name, o in (("threshold", dict(policy="threshold")), ("pull", dict(policy="forced", forced_mode="pull")),
                        ("push_dense", dict(policy="forced", forced_mode="push_dense")),
                        ("push_sparse", dict(policy="forced", forced_mode="push_sparse")),
                        ("mlp", dict(policy="mlp"))):
            try:
                ts = [G.run(app, stream=stream, **o).elapsed_ms for _ in range(3)]
                pol[name] = round(min(ts), 4)
            except ipg.IPError:
                pol[name] = None
        detail[app]["policy_ms"] = pol
    # PageRank at the small configuration (R-MAT scale 16, directed, T = 30)
    import inputs
    pg = inputs.rmat_graph(16, seed=1)
    with ipg.Graph.from_inputs(pg, stream=stream) as P:
        ts = [P.run("pagerank", stream=stream, policy="forced", forced_mode="pull").elapsed_ms for _ in range(5)]
        pr_ms = min(ts)
    detail["pagerank_scale16"] = {"gteps": round(30 * pg.m / (pr_ms * 1e-3) / 1e9, 2), "ms": round(pr_ms, 4),
                                  "edges": pg.m}
    G.close()
    return dict(value=value, total_ms=total_ms, msgs=msgs_all, launches=launches, roofline=roofline,
                e2e=dict(value=round(e2e_value, 3), unit="GTEPS", h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h,
                         median_step_ms=round(statistics.median(e2e_ms), 3)),
                clocks=clk.summary(), detail=detail, V=V, E=E, kernels={k: [round(v[0], 3), v[2]] for k, v in kern.items()})


# ----------------------------------------------------------------- CPU oracle (baseline and reference arm)
def oracle_step(g):
    import oracle
    t0 = time.perf_counter()
    _, a = oracle.hashmin(g.n, g.row_ptr, g.col)
    _, b = oracle.sssp(g.n, g.row_ptr, g.col, g.w, source=0)
    dt = time.perf_counter() - t0
    return int(a["messages"].sum()) + int(b["messages"].sum()), dt


def cpu_oracle_pagerank(g, T, sample):
    """The FP64 oracle's PageRank on the host cores (single-threaded), GTEPS = T*E / s."""
    import oracle
    t0 = time.perf_counter()
    oracle.pagerank(g.n, g.row_ptr, g.col, T=T)
    dt = time.perf_counter() - t0
    return {"value": round(T * g.m / dt / 1e9, 5), "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": sample,
            "seconds": round(dt, 2)}


def cpu_baseline(g):
    m, dt = oracle_step(g)
    return {"value": round(m / dt / 1e9, 5), "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": "one full step: Hashmin + SSSP(source 0) on the same scale-22 graph, single-threaded",
            "seconds": round(dt, 2)}


def run_reference(args):
    g = build_graph(args.scale)
    for _ in range(args.warmup):  # warm-up: the Hashmin half of a step (the oracle has no state to warm)
        import oracle
        oracle.hashmin(g.n, g.row_ptr, g.col)
    msgs, secs = 0, 0.0
    for _ in range(args.steps):
        m, dt = oracle_step(g)
        msgs += m
        secs += dt
    value = msgs / secs / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "GTEPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * secs / args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "scale": args.scale, "policy": "oracle (push, literal Pregel)"},
            "cpu_baseline": {"value": round(value, 5), "unit": "GTEPS", "cores": 1, "kind": "oracle",
                             "sample": "every step: Hashmin + SSSP(source 0) on the full scale-22 graph"},
            "e2e": {"value": round(value, 5), "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def ncu_case(spec, scale):
    """Small profiling case: one app in one forced mode, host-driven loop (ncu cannot
    profile kernels inside graphs with conditional nodes), run twice; or
    batch_sssp:K — K sources at once in the persistent kernel."""
    import paper_2010_08781_gb300 as ipg
    app, mode, *rest = spec.split(":")
    if app == "pagerank":  # directed R-MAT, as the PageRank configurations use
        import inputs
        g = inputs.rmat_graph(scale, edge_factor=EDGE_FACTOR, a=0.57, b=0.19, c=0.19, seed=1)
    else:
        g = build_graph(scale)
    if app == "batch_sssp":
        import inputs
        k = int(mode)
        src = np.concatenate([[0], inputs.uniform_vertices(g.n, k - 1, seed=1)]).astype(np.uint32)
        with ipg.Graph.from_inputs(g) as G:
            for _ in range(2):
                _, st = G.run_batch_sssp(src)
        print(json.dumps({"ncu_case": spec, "scale": scale, "edges": g.m, "supersteps": st["supersteps"],
                          "ms": round(st["elapsed_ms"], 4), "messages": st["messages"]}))
        return
    with ipg.Graph.from_inputs(g) as G:
        for _ in range(2):
            kw = dict(policy="forced", forced_mode=mode) if app != "pagerank" or mode != "auto" else {}
            if rest:  # PageRank pull engine: gather or blocked
                kw["pr_engine"] = rest[0]
            st = G.run(app, use_graph=0, **kw)
    print(json.dumps({"ncu_case": spec, "scale": scale, "edges": g.m, "supersteps": st.supersteps,
                      "ms": round(st.elapsed_ms, 4)}))


def pr_measure(G, V, E, reps=3, T=30, engine="auto"):
    """PageRank pull, T iterations: device time of the run and the roofline of its
    pull exchange (the CSC gather k_pr_pull, or the blocked pull's two launches
    k_pb_scatter + k_pb_accumulate): algorithmic bytes 8E + 16V + 4(V+1) per
    superstep (in-edge indices and their sources' broadcasts; offsets, ranks,
    broadcasts, out-degrees) over the exchange time, CUDA events per superstep."""
    peak, kind = measured_peaks()
    kw = dict(policy="forced", forced_mode="pull", pr_iterations=T, pr_engine=engine)
    ts = [G.run("pagerank", **kw).elapsed_ms for _ in range(reps)]
    st = G.run("pagerank", profile_kernels=1, **kw)
    kms = [float(x) for x in st.kernel_ms[1:st.supersteps, 1]]
    by = 4 * (V + 1) + 8 * E + 16 * V
    avg = sum(kms) / len(kms)
    ach = by / (avg * 1e-3) / 1e9
    blocked = engine == "blocked" or (engine == "auto" and E >= 1 << 24)
    kern = "k_pb_scatter+k_pb_accumulate" if blocked else "k_pr_pull"
    return {"engine": "blocked" if blocked else "gather", "gteps": round(T * E / (min(ts) * 1e-3) / 1e9, 2),
            "ms": round(min(ts), 4), "ms_per_iteration": round(min(ts) / T, 4),
            "roofline": {"bound": "hbm", "kernel": kern, "achieved": round(ach, 1), "peak": peak,
                         "peak_kind": kind, "unit": "GB/s", "frac": round(ach / peak, 4),
                         "traffic": measured_traffic(kern) if E >= 10**9 else None,  # captured at scale 26
                         "avg_launch_us": round(1e3 * avg, 2), "bytes_per_launch": by}}


def run_config(args):
    """Secondary measured configurations (one JSON line each)."""
    import paper_2010_08781_gb300 as ipg
    import inputs
    import torch
    torch.cuda.set_device(0)
    out = {"config": args.config}
    if args.config == "c1":  # PageRank, directed R-MAT scale 16, T = 30
        g = inputs.rmat_graph(16, seed=1)
        with ipg.Graph.from_inputs(g) as G:
            out["pagerank"] = pr_measure(G, g.n, g.m)
        out["cpu_oracle"] = cpu_oracle_pagerank(g, 30, "PageRank T=30 on the full graph")
        out["workload"] = "PageRank T=30 on directed R-MAT scale 16 (edge factor 16, seed 1)"
        out["edges"] = g.m
    elif args.config == "c4":  # batched
        g = inputs.rmat_graph(20, symmetrize=True, weighted=True, seed=1)
        src = np.concatenate([[0], inputs.uniform_vertices(g.n, 255, seed=1)]).astype(np.uint32)
        with ipg.Graph.from_inputs(g) as G:
            G.run_batch_sssp(src)
            rs = [G.run_batch_sssp(src)[1] for _ in range(3)]
            seq = [G.run("sssp", source=int(s)).elapsed_ms for s in src[:32]]
        best = min(r["elapsed_ms"] for r in rs)
        out["batch_sssp"] = {"sources": 256, "ms": round(best, 3), "supersteps": rs[0]["supersteps"],
                             "messages": rs[0]["messages"],
                             "gteps": round(rs[0]["messages"] / (best * 1e-3) / 1e9, 2),
                             "sequential_ms_estimate": round(sum(seq) * 256 / 32, 2)}
        del g
        gs = inputs.hashmin_instances(1000, seed=1)
        u, offs = inputs.block_diagonal(gs)
        with ipg.Graph.from_inputs(u) as G:
            G.run_batch_hashmin(offs.astype(np.uint32))
            rs = [G.run_batch_hashmin(offs.astype(np.uint32))[1] for _ in range(3)]
            pers = min(G.run_batch_hashmin(offs.astype(np.uint32), engine="persistent")[1]["elapsed_ms"]
                       for _ in range(3))
            single = min(G.run("hashmin").elapsed_ms for _ in range(3))
        best = min(r["elapsed_ms"] for r in rs)
        out["batch_hashmin"] = {"instances": 1000, "vertices": u.n, "edges": u.m, "ms": round(best, 3),
                                "supersteps": rs[0]["supersteps"], "messages": rs[0]["messages"],
                                "gteps": round(rs[0]["messages"] / (best * 1e-3) / 1e9, 2),
                                "persistent_engine_ms": round(pers, 3), "ip_run_union_ms": round(single, 3)}
        out["workload"] = ("256 SSSP sources on symmetrised weighted R-MAT scale 20; 1,000 Hashmin instances, "
                           "R-MAT 1k-100k vertices (log-uniform), edge factor 8, symmetrised")
    elif args.config == "c5":  # billion-edge
        g = inputs.rmat_graph(26, seed=1)
        V, E = g.n, g.m
        out["cpu_oracle_pagerank"] = cpu_oracle_pagerank(g, 1, "PageRank with T=1 (one rank update) on the full graph")
        with ipg.Graph(V, g.row_ptr, g.col) as G:  # in-edges transposed on the device
            del g
            out["pagerank"] = pr_measure(G, V, E, reps=2)
            out["pagerank"]["vertices"], out["pagerank"]["edges"] = V, E
            out["pagerank_gather"] = pr_measure(G, V, E, reps=2, engine="gather")
        src, dst = inputs.rmat_edges(26, 16 << 26, seed=1)
        gs = inputs.from_edges(1 << 26, src, dst, symmetrize=True)
        del src, dst
        with ipg.Graph.from_inputs(gs) as G:
            ts = [G.run("hashmin") for _ in range(2)]
        best = min(ts, key=lambda r: r.elapsed_ms)
        m = int(best.messages.sum())
        out["hashmin_symmetrised"] = {"vertices": gs.n, "edges": gs.m, "ms": round(best.elapsed_ms, 3),
                                      "supersteps": best.supersteps, "gteps": round(m / (best.elapsed_ms * 1e-3) / 1e9, 2),
                                      "modes": best.mode[1:].tolist()}
        out["workload"] = "R-MAT scale 26, edge factor 16, seed 1: PageRank T=30 pull (directed), Hashmin (symmetrised)"
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--scale", type=int, default=SCALE)
    ap.add_argument("--policy", default="auto")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ncu-case", default=None,
                    help="APP:MODE[:ENGINE], e.g. sssp:pull or pagerank:pull:blocked — small profiling case only")
    ap.add_argument("--config", default=None, choices=["c1", "c4", "c5"],
                    help="secondary configurations: c1 PageRank scale 16, c4 batched, c5 scale 26")
    args = ap.parse_args()
    if args.config:
        run_config(args)
        return
    if args.ncu_case:
        ncu_case(args.ncu_case, args.scale)
        return
    args.warmup = max(args.warmup, 3) if args.impl == "gb300" else args.warmup

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return
    if world > 1:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    r = run_gpu(args, rank, world, local_rank)
    if rank == 0:
        line = {"metric": METRIC, "value": round(r["value"], 3), "unit": "GTEPS", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(r["total_ms"] / args.steps, 4),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "scale": args.scale, "vertices": r["V"], "edges": r["E"],
                           "policy": args.policy, "l2": "flushed between timed steps; inputs (1.03 GB) exceed L2",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "roofline": r["roofline"], "e2e": r["e2e"], "gpu_launches": r["launches"], "clocks": r["clocks"],
                "per_app": r["detail"], "kernel_ms_by_name": r["kernels"]}
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(build_graph(args.scale))
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
