#!/usr/bin/env python3
"""Benchmark of the synchronous vertex-centric superstep library on one GB300.

Default workload (one "step"): the billion-edge configuration — directed R-MAT
scale 26 (67,108,864 vertices, edge factor 16, (a,b,c,d) = (.57,.19,.19,.05),
seed 1, duplicates removed: 1,060,392,804 edges), PageRank with T = 30 rank
updates in pull (blocked pull engine), plus Hashmin connected components on the
symmetrised form of the same edges (2,103,866,764 directed edges), each run to
global halt.

Metric: GTEPS = edges traversed by messages (PageRank: E per broadcasting
superstep, T·E per run; Hashmin: the out-degrees of the broadcasting vertices,
summed over supersteps) / step time; per app, gteps_graph500 is the graph's edge
count over the run time. The JSON line also carries the roofline of
the dominant kernel (the blocked pull's two launches per superstep: 8E + 20V
algorithmic bytes over their CUDA-event time, against the measured HBM copy
bandwidth), the end-to-end number through the C ABI from pinned host buffers,
the device memory footprint, and the CPU oracle timed on the host cores. The
secondary configurations (Hashmin + SSSP on symmetrised R-MAT 22, PageRank on
R-MAT 16) are reported under per_app.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
  python bench.py --config c2|c1|c4|bfs_perm   secondary configurations, one line each
  python bench.py --ncu-case APP:MODE[:ENGINE] --scale S   small profiling case
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

SCALE = 26
EDGE_FACTOR = 16
T_PR = 30
C2_SCALE = 22
METRIC = "GTEPS & % HBM BW per app (PageRank/Hashmin/SSSP); learned vs fixed push/pull"
WORKLOAD = ("billion-edge: PageRank T=30 pull on directed R-MAT scale 26 (edge factor 16, "
            "(a,b,c,d)=(.57,.19,.19,.05), seed 1, duplicates removed) + Hashmin on its symmetrised form")
C2_WORKLOAD = ("Hashmin + SSSP(source 0) on symmetrised R-MAT scale 22, edge factor 16, "
               "(a,b,c,d)=(.57,.19,.19,.05), seed 1, duplicates removed, uint32 weights in [1,255]")
L2_BYTES = 129 * 1024 * 1024


def c2_graph(scale=C2_SCALE):
    import inputs
    return inputs.rmat_graph(scale, edge_factor=EDGE_FACTOR, a=0.57, b=0.19, c=0.19, seed=1, symmetrize=True,
                             weighted=True, wseed=1)


def c5_graphs(scale=SCALE, symmetric=True):
    """The directed R-MAT graph (with its host CSC) and, if asked, its symmetrised form."""
    import inputs
    src, dst = inputs.rmat_edges(scale, EDGE_FACTOR << scale, 0.57, 0.19, 0.19, 1)
    d = inputs.from_edges(1 << scale, src, dst)
    s = inputs.from_edges(1 << scale, src, dst, symmetrize=True) if symmetric else None
    return d, s


def stored_traffic(kernel):
    """DRAM bytes per launch of a kernel from profiles/traffic.json: an ncu capture
    (dram__bytes_read.sum + dram__bytes_write.sum) on a small case, scaled to the
    benchmark's workload by the edges processed. A stored profile figure, not a
    measurement of this run; None when the kernel has no capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel)
    return None if e is None else e.get("bytes_per_launch_at_benchmark_size")


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


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
def launches_of(mode_seq, app, blocked=False):
    """Kernels one run launches: superstep 0 (PageRank: k_pr_init; a vertex program:
    k_ctl_init + k_init_prog) + the selector, then per superstep the mode's kernels +
    the selector (blocked: the pull streams the blocked layout, two kernels)."""
    n = 2 if app == "pagerank" else 3
    for m in mode_seq[1:]:
        if app == "pagerank":
            n += (3 if blocked else 2) if m == 2 else 3
        elif m == 0:
            n += 4  # compaction, push, apply, selector
        else:
            n += 4 if (m == 2 and blocked) else 3  # (scatter + accumulate | pull | push), apply, selector
    return n


def pr_pull_bytes(V, E):
    """Algorithmic bytes of one PageRank pull superstep: 4E in-edge indices + 4E
    gathered source broadcasts + 20V (offsets, rank write, broadcast write,
    out-degree, sum) = 8E + 20V."""
    return 8 * E + 20 * V


def exchange_bytes(app, mode, V, E, active_sources, bcast_prev, recipients, weighted_edges=0):
    """Algorithmic bytes of one min-app exchange launch delivering the broadcasts of
    the previous superstep.

    pull:  4E in-edge sources (+ 4E in-edge weights, SSSP) + 4 per gathered active
           source + 16V (offsets, mailbox, broadcast slot, recipient and broadcast bits)
    push:  16 per sender (offsets, value, queue entry or bitmap word) + per message
           (8 Hashmin / 12 SSSP: target, weight, the combining RMW counted once) + 20 per
           recipient."""
    w = 4 if app == "sssp" else 0
    if mode == 2:
        return 4 * E + w * E + 4 * active_sources + 16 * V
    per_msg = 8 + w
    return 16 * bcast_prev + per_msg * active_sources + 20 * recipients


KERNEL_NAMES = {("pull", "hashmin"): "k_pull<Hashmin>", ("pull", "sssp"): "k_pull<SSSP>",
                ("push_dense", "hashmin"): "k_push<Hashmin,dense>", ("push_dense", "sssp"): "k_push<SSSP,dense>",
                ("push_sparse", "hashmin"): "k_push<Hashmin,sparse>",
                ("push_sparse", "sssp"): "k_push<SSSP,sparse>"}
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


# ----------------------------------------------------------------- CPU oracle pool
# One superstep of each app by the oracle (oracle.pagerank_superstep on the directed
# graph, oracle.hashmin_superstep on the symmetrised one: FP64 / uint32, plain loops),
# statically partitioned over the host cores: every worker process takes a
# contiguous range of vertices (the paper's static OpenMP schedule over vertices),
# the graphs shared through shared memory. The oracle itself is unchanged.
_W = {}


def _pool_attach(spec):
    from multiprocessing import shared_memory
    import oracle
    oracle.build()
    arrs = {}
    for name, (shm_name, dtype, count) in spec.items():
        shm = shared_memory.SharedMemory(name=shm_name)
        _W.setdefault("shm", []).append(shm)
        arrs[name] = np.ndarray((count,), dtype=np.dtype(dtype), buffer=shm.buf)
    _W["a"] = arrs


def _pool_task(task):
    import oracle
    a = _W["a"]
    kind, v0, v1 = task
    n = int(a["n"][0])
    if v1 <= v0:
        return 0
    if kind == "pagerank":
        a["pr_out"][v0:v1] = oracle.pagerank_superstep(n, a["d_ptr"], a["d_idx"], a["outdeg"], a["prev"], 0.85,
                                                       v0, v1)
    else:
        a["hm_out"][v0:v1] = oracle.hashmin_superstep(n, a["s_ptr"], a["s_idx"], a["label"], a["bcast"], v0, v1)
    return v1 - v0


class OraclePool:
    """Spawned worker processes (no fork after CUDA use) running one oracle superstep
    of PageRank (directed graph d) and of Hashmin (symmetrised graph s, superstep 1:
    every vertex broadcast its id in superstep 0) on disjoint vertex ranges."""

    def __init__(self, d, s, workers):
        import multiprocessing as mp
        from multiprocessing import shared_memory
        self.n, self.workers = d.n, workers
        src = {"n": np.array([d.n], np.uint32), "d_ptr": d.t_ptr, "d_idx": d.t_idx,
               "outdeg": d.out_degree().astype(np.uint32), "prev": np.full(d.n, 1.0 / d.n),
               "pr_out": np.zeros(d.n, np.float64)}
        if s is not None:
            src.update({"s_ptr": s.t_ptr, "s_idx": s.t_idx, "label": np.arange(s.n, dtype=np.uint32),
                        "bcast": np.ones(s.n, np.uint8), "hm_out": np.zeros(s.n, np.uint32)})
        self.shm, spec = [], {}
        for name, arr in src.items():
            arr = np.ascontiguousarray(arr)
            shm = shared_memory.SharedMemory(create=True, size=max(arr.nbytes, 8))
            np.ndarray(arr.shape, arr.dtype, buffer=shm.buf)[:] = arr
            self.shm.append(shm)
            spec[name] = (shm.name, arr.dtype.str, arr.size)
        self.ptr = {"pagerank": d.t_ptr, "hashmin": s.t_ptr if s is not None else None}
        self.pool = mp.get_context("spawn").Pool(workers, initializer=_pool_attach, initargs=(spec,))
        self.pool.map(_pool_task, [("pagerank", 0, 0)] * workers)  # workers up and attached

    def superstep(self, kind, v_begin=0, v_end=None, parts=None):
        """Seconds for one oracle superstep of `kind` over [v_begin, v_end), split into
        `parts` equal vertex ranges (default: one per worker)."""
        v_end = self.n if v_end is None else v_end
        parts = self.workers if parts is None else parts
        cuts = np.linspace(v_begin, v_end, parts + 1).astype(np.int64)
        t0 = time.perf_counter()
        self.pool.map(_pool_task, [(kind, int(cuts[i]), int(cuts[i + 1])) for i in range(parts)], chunksize=1)
        return time.perf_counter() - t0

    def edges(self, kind, v_begin=0, v_end=None):
        v_end = self.n if v_end is None else v_end
        return int(self.ptr[kind][v_end]) - int(self.ptr[kind][v_begin])

    def step(self):
        """One sample of the default step: a PageRank and a Hashmin superstep over
        every vertex; (edges, seconds)."""
        kinds = ("pagerank", "hashmin") if self.ptr["hashmin"] is not None else ("pagerank",)
        t = sum(self.superstep(k) for k in kinds)
        return sum(self.edges(k) for k in kinds), t

    def close(self):
        self.pool.close()
        self.pool.join()
        for s in self.shm:
            s.close()
            s.unlink()


SAMPLE = ("one PageRank superstep (Fig. 8, FP64, oracle.pagerank_superstep) over the {ed:,} edges of the directed "
          "graph and one Hashmin superstep (Fig. 9, superstep 1, oracle.hashmin_superstep) over the {es:,} edges of "
          "the symmetrised graph, every vertex, static vertex ranges over {w} host cores")


def cpu_oracle_baseline(pool, d, s):
    """The oracle's supersteps on the host: all cores (static vertex ranges, one per
    core) over both whole graphs, and one core over a slice of the directed graph."""
    best = min((pool.step() for _ in range(2)), key=lambda x: x[1])
    edges, secs = best
    all_cores = {"value": round(edges / secs / 1e9, 5), "unit": "GTEPS", "cores": pool.workers, "kind": "oracle",
                 "sample": SAMPLE.format(ed=d.m, es=s.m, w=pool.workers), "seconds": round(secs, 3),
                 "host_cores": host_cores()}
    v1 = int(np.searchsorted(d.t_ptr, d.m // 8))  # about an eighth of the directed edges
    t1 = pool.superstep("pagerank", 0, v1, parts=1)
    all_cores["single_thread"] = {"value": round(pool.edges("pagerank", 0, v1) / t1 / 1e9, 5), "unit": "GTEPS",
                                  "cores": 1, "seconds": round(t1, 3),
                                  "sample": f"the PageRank superstep for vertices [0, {v1:,}) "
                                            f"({pool.edges('pagerank', 0, v1):,} edges)"}
    return all_cores


# ----------------------------------------------------------------- GPU arm
def memory_report(G, name):
    info = G.info()
    V, E = info["n_vertices"], info["n_edges"]
    rep = {"graph": name, "vertices": V, "edges": E, "device_bytes": info["device_bytes"],
           "bytes_per_vertex": round(info["device_bytes"] / V, 2), "bytes_per_edge": round(info["device_bytes"] / E, 3)}
    parts = {k[len("bytes_"):]: info[k] for k in info if k.startswith("bytes_") and info[k]}
    if parts:
        rep["breakdown"] = parts
    return rep


def run_gpu(args, rank, world, local_rank):
    import torch
    import paper_2010_08781_gb300 as ipg

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    d, s = c5_graphs(args.scale)
    V, Ed, Es = d.n, d.m, s.m
    # the CPU oracle's workers are spawned (not forked) and stay idle until the GPU legs are done
    pool = OraclePool(d, s, host_cores()) if rank == 0 and world == 1 and not args.no_cpu_baseline else None
    # pinned host copies of the inputs (the end-to-end leg copies them every step)
    pin = {k: torch.from_numpy(v.view(np.int32)).pin_memory()
           for k, v in (("d_ptr", d.row_ptr), ("d_col", d.col), ("s_ptr", s.row_ptr), ("s_col", s.col))}
    with torch.cuda.stream(stream):
        P = ipg.Graph(V, pin["d_ptr"], pin["d_col"], stream=stream)  # in-edges transposed on the device
        H = ipg.Graph(V, pin["s_ptr"], pin["s_col"], symmetric=True, stream=stream)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    pr_kw = dict(policy="forced", forced_mode="pull", pr_iterations=T_PR, stream=stream)
    hm_kw = dict(policy=args.policy, stream=stream)

    def step():
        return P.run("pagerank", **pr_kw), H.run("hashmin", **hm_kw)

    clk = ClockSampler(local_rank).__enter__()  # sampling from before the warm-up
    for _ in range(args.warmup):
        step()  # the first one also builds the blocked layout
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    msgs = launches = 0
    runs = {"pagerank": [], "hashmin": []}
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
            hm_blocked = H.info()["bytes_blocked_layout"] > 0  # built at the start of a run that uses it
            launches += (launches_of(a.mode.tolist(), "pagerank", blocked=True) +
                         launches_of(b.mode.tolist(), "hashmin", blocked=hm_blocked))
            runs["pagerank"].append(a)
            runs["hashmin"].append(b)
        torch.cuda.synchronize()
    finally:
        clk.stop()
        clk.__exit__(None, None, None)
    step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    total_ms, msgs_all = reduce_over_ranks(sum(step_ms), msgs, world, dev)
    value = msgs_all / (total_ms * 1e-3) / 1e9

    # ---------------------------------------------------------- roofline of the dominant kernel
    # Host-driven replay of the timed PageRank runs (same engine, same graph state), CUDA
    # events on the launching stream around the two blocked-pull launches of every superstep.
    peak, peak_kind = measured_peaks()
    by = pr_pull_bytes(V, Ed)
    pull_ms = []
    for _ in range(min(args.steps, 3)):
        st = P.run("pagerank", profile_kernels=1, **pr_kw)
        pull_ms += [float(x) for x in st.kernel_ms[1:st.supersteps, 1]]
    avg = sum(pull_ms) / len(pull_ms)
    achieved = by / (avg * 1e-3) / 1e9
    pr_ms = statistics.median(r.elapsed_ms for r in runs["pagerank"])
    hm_ms = statistics.median(r.elapsed_ms for r in runs["hashmin"])
    roofline = {"bound": "hbm", "kernel": "k_pb_scatter+k_pb_accumulate", "achieved": round(achieved, 1),
                "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": stored_traffic("k_pb_scatter+k_pb_accumulate"),
                "traffic_note": ("stored ncu figure (profiles/traffic.json: R-MAT 23 capture scaled by edges), "
                                 "not measured in this run"),
                "bytes_per_launch": by, "launches_per_step": T_PR, "avg_launch_us": round(1e3 * avg, 2),
                "timing": "CUDA events per superstep around the pull launches, host-driven replay after the timed region",
                "timed_region_lower_bound_gbs": round(by * T_PR / (pr_ms * 1e-3) / 1e9, 1),
                "share_of_step": round(T_PR * avg / (pr_ms + hm_ms), 3)}

    # ---------------------------------------------------------- per app, policies, memory
    detail = {}
    pm = int(runs["pagerank"][0].messages.sum())
    detail["pagerank"] = {"gteps": round(pm / (pr_ms * 1e-3) / 1e9, 2), "ms": round(pr_ms, 3),
                          "ms_per_iteration": round(pr_ms / T_PR, 4), "supersteps": runs["pagerank"][0].supersteps,
                          "vertices": V, "edges": Ed, "engine": "blocked"}
    gather = min(P.run("pagerank", pr_engine="gather", **pr_kw).elapsed_ms for _ in range(2))
    detail["pagerank"]["gather_engine_ms"] = round(gather, 3)
    hmsg = int(runs["hashmin"][0].messages.sum())
    detail["hashmin"] = {"gteps": round(hmsg / (hm_ms * 1e-3) / 1e9, 2),
                         "gteps_graph500": round(Es / (hm_ms * 1e-3) / 1e9, 2), "ms": round(hm_ms, 3),
                         "supersteps": runs["hashmin"][0].supersteps, "messages": hmsg, "edges": Es,
                         "modes": runs["hashmin"][0].mode[1:].tolist(),
                         "policy_ms": policy_times(H, "hashmin", stream, ipg)}
    memory = [memory_report(P, "directed R-MAT 26 (PageRank, blocked layout built)"),
              memory_report(H, "symmetrised R-MAT 26 (Hashmin)")]
    P.close()
    H.close()

    # ---------------------------------------------------------- end to end through the C ABI, host buffers
    e2e_steps = max(1, min(args.steps, 5))
    out_f = torch.empty(V, dtype=torch.float32).pin_memory()
    out_u = torch.empty(V, dtype=torch.int32).pin_memory()
    e2e_ms = []
    phases = {k: [] for k in ("create_directed", "pagerank_run", "pagerank_device", "values_pagerank",
                              "destroy_directed", "create_symmetrised", "hashmin_run", "hashmin_device",
                              "values_hashmin", "destroy_symmetrised")}

    def lap(name, t):
        torch.cuda.synchronize()
        now = time.perf_counter()
        phases[name].append(1e3 * (now - t))
        return now

    for i in range(e2e_steps):
        torch.cuda.synchronize()
        t0 = t = time.perf_counter()
        A = ipg.Graph(V, pin["d_ptr"], pin["d_col"], stream=stream)
        t = lap("create_directed", t)
        ra = A.run("pagerank", **pr_kw)
        t = lap("pagerank_run", t)
        A.values(out=out_f, stream=stream)
        t = lap("values_pagerank", t)
        A.close()
        t = lap("destroy_directed", t)
        B = ipg.Graph(V, pin["s_ptr"], pin["s_col"], symmetric=True, stream=stream)
        t = lap("create_symmetrised", t)
        rb = B.run("hashmin", **hm_kw)
        t = lap("hashmin_run", t)
        B.values(out=out_u, stream=stream)
        t = lap("values_hashmin", t)
        B.close()
        t = lap("destroy_symmetrised", t)
        phases["pagerank_device"].append(ra.elapsed_ms)
        phases["hashmin_device"].append(rb.elapsed_ms)
        e2e_ms.append(1e3 * (t - t0))
    h2d = 4 * (V + 1) + 4 * Ed + 4 * (V + 1) + 4 * Es
    e2e = {"value": round((msgs / args.steps) / (statistics.median(e2e_ms) * 1e-3) / 1e9, 3), "unit": "GTEPS",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 2 * 4 * V, "steps": e2e_steps,
           "median_step_ms": round(statistics.median(e2e_ms), 2),
           "phases_median_ms": {k: round(statistics.median(v), 2) for k, v in phases.items()},
           "covers": "graph creation from pinned host CSR (device transposition, renumbering, degree bins, "
                     "blocked layout), both runs, results copied to pinned host memory, destroy"}
    del pin
    ipg.release_cached_memory()

    # ---------------------------------------------------------- secondary configurations
    detail["c2_scale22"] = c2_summary(args, stream, ipg)
    detail["c1_pagerank_scale16"] = c1_summary(stream, ipg)
    cpu = None
    if pool is not None:
        cpu = cpu_oracle_baseline(pool, d, s)
        pool.close()
    return dict(value=value, total_ms=total_ms, launches=launches, roofline=roofline, e2e=e2e,
                clocks=clk.summary(), detail=detail, V=V, Ed=Ed, Es=Es, memory=memory, cpu=cpu)


def policy_times(G, app, stream, ipg, reps=3):
    """Best of reps whole-run times per policy, and the modes the two selectors chose."""
    pol, modes = {}, {}
    for name, o in (("threshold", dict(policy="threshold")), ("mlp", dict(policy="mlp")),
                    ("pull", dict(policy="forced", forced_mode="pull")),
                    ("push_dense", dict(policy="forced", forced_mode="push_dense")),
                    ("push_sparse", dict(policy="forced", forced_mode="push_sparse"))):
        try:
            rs = [G.run(app, stream=stream, **o) for _ in range(reps)]
            pol[name] = round(min(r.elapsed_ms for r in rs), 4)
            if name in ("threshold", "mlp"):
                modes[name] = rs[0].mode[1:].tolist()
        except ipg.IPError:
            pol[name] = None
    pol["modes"] = modes
    return pol


def c2_summary(args, stream, ipg, steps=10):
    g = c2_graph()
    out = {"workload": C2_WORKLOAD, "vertices": g.n, "edges": g.m}
    with ipg.Graph.from_inputs(g, stream=stream) as G:
        for app, kw in (("hashmin", {}), ("sssp", dict(source=0))):
            rs = [G.run(app, policy=args.policy, stream=stream, **kw) for _ in range(steps + 2)][2:]
            ms = statistics.median(r.elapsed_ms for r in rs)
            m = int(rs[0].messages.sum())
            out[app] = {"gteps": round(m / (ms * 1e-3) / 1e9, 2), "gteps_graph500": round(g.m / (ms * 1e-3) / 1e9, 2),
                        "ms": round(ms, 4), "supersteps": rs[0].supersteps,
                        "messages": m, "modes": rs[0].mode[1:].tolist(),
                        "policy_ms": policy_times(G, app, stream, ipg)}
        out["memory"] = memory_report(G, "symmetrised weighted R-MAT 22")
    tot = out["hashmin"]["ms"] + out["sssp"]["ms"]
    out["gteps_step"] = round((out["hashmin"]["messages"] + out["sssp"]["messages"]) / (tot * 1e-3) / 1e9, 2)
    return out


def c1_summary(stream, ipg):
    import inputs
    pg = inputs.rmat_graph(16, seed=1)
    with ipg.Graph.from_inputs(pg, stream=stream) as P:
        ts = [P.run("pagerank", stream=stream, policy="forced", forced_mode="pull").elapsed_ms for _ in range(5)]
        mem = memory_report(P, "directed R-MAT 16")
    pr_ms = min(ts)
    return {"gteps": round(30 * pg.m / (pr_ms * 1e-3) / 1e9, 2), "ms": round(pr_ms, 4), "edges": pg.m,
            "memory": mem}


# ----------------------------------------------------------------- reference arm (the CPU oracle)
def run_reference(args):
    d, sg = c5_graphs(args.scale)
    pool = OraclePool(d, sg, host_cores())
    for _ in range(args.warmup):
        pool.step()
    steps = [pool.step() for _ in range(args.steps)]
    pool.close()
    edges, secs = sum(e for e, _ in steps), sum(t for _, t in steps)
    value = edges / secs / 1e9
    sample = "every step: " + SAMPLE.format(ed=d.m, es=sg.m, w=pool.workers)
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "GTEPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * secs / args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "scale": args.scale, "vertices": d.n, "edges_directed": d.m,
                       "edges_symmetrised": sg.m, "policy": "oracle (literal Pregel supersteps)"},
            "cpu_baseline": {"value": round(value, 5), "unit": "GTEPS", "cores": pool.workers, "kind": "oracle",
                             "sample": sample, "host_cores": host_cores()},
            "e2e": {"value": round(value, 5), "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- secondary configurations
def ncu_case(spec, scale):
    """Small profiling case: one app in one forced mode, host-driven loop (ncu cannot
    profile kernels inside graphs with conditional nodes), run twice; or
    batch_sssp:K — K sources at once in the persistent kernel."""
    import paper_2010_08781_gb300 as ipg
    if spec == "default":  # the default line's workload, one step, host-driven (every launch visible to ncu)
        d, sg = c5_graphs(scale)
        out = {"ncu_case": spec, "scale": scale}
        with ipg.Graph(d.n, d.row_ptr, d.col) as P:
            del d
            st = P.run("pagerank", policy="forced", forced_mode="pull", pr_iterations=T_PR, use_graph=0)
            out["pagerank_ms"] = round(st.elapsed_ms, 3)
        with ipg.Graph(sg.n, sg.row_ptr, sg.col, symmetric=True) as H:
            st = H.run("hashmin", use_graph=0)
            out["hashmin_ms"] = round(st.elapsed_ms, 3)
            out["hashmin_modes"] = st.mode[1:].tolist()
        print(json.dumps(out))
        return
    app, mode, *rest = spec.split(":")
    if app == "pagerank":  # directed R-MAT, as the PageRank configurations use
        import inputs
        g = inputs.rmat_graph(scale, edge_factor=EDGE_FACTOR, a=0.57, b=0.19, c=0.19, seed=1)
    else:
        g = c2_graph(scale)
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


def c2_line(args, steps):
    """The Hashmin + SSSP configuration on its own line, with the roofline of its
    dominant kernel (per-kernel CUDA events in a host-driven replay of the timed
    runs' mode sequences)."""
    import torch
    import paper_2010_08781_gb300 as ipg
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    g = c2_graph(args.scale if args.scale != SCALE else C2_SCALE)
    V, E = g.n, g.m
    with ipg.Graph.from_inputs(g, stream=stream) as G:
        def step():
            return G.run("hashmin", policy=args.policy, stream=stream), G.run("sssp", policy=args.policy,
                                                                                stream=stream)
        for _ in range(3):
            step()
        clk = ClockSampler(0).__enter__()
        torch.cuda.synchronize()
        clk.start()
        rs = [step() for _ in range(steps)]
        torch.cuda.synchronize()
        clk.stop()
        clk.__exit__(None, None, None)
        ms = sum(a.elapsed_ms + b.elapsed_ms for a, b in rs)
        msgs = sum(int(a.messages.sum()) + int(b.messages.sum()) for a, b in rs)
        kern = {}
        peak, kind = measured_peaks()
        blocked = G.info()["bytes_blocked_layout"] > 0  # AUTO pulls on the layout once it exists
        for app, last in (("hashmin", rs[-1][0]), ("sssp", rs[-1][1])):
            seq = last.mode[1:last.supersteps].tolist()
            st = G.run(app, profile_kernels=1, stream=stream, mode_sequence=seq)
            for s in range(1, st.supersteps):
                mode = int(st.mode[s])
                name = KERNEL_NAMES[(MODE_NAMES[mode], app)]
                if blocked and MODE_NAMES[mode] == "pull":
                    name = f"k_pbm_scatter+k_pbm_accumulate ({app})"
                by = exchange_bytes(app, mode, V, E, int(st.messages[s - 1]), int(st.broadcasters[s - 1]),
                                    int(st.active[s]))
                k = kern.setdefault(name, [0.0, 0.0, 0])
                k[0] += float(st.kernel_ms[s, 1])
                k[1] += by
                k[2] += 1
        dom = max(kern, key=lambda n: kern[n][0])
        d_ms, d_by, d_n = kern[dom]
        ach = d_by / (d_ms * 1e-3) / 1e9
        line = {"config": "c2", "workload": C2_WORKLOAD, "vertices": V, "edges": E,
                "gteps": round(msgs / (ms * 1e-3) / 1e9, 3), "ms_per_step": round(ms / steps, 4),
                "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(ach, 1), "peak": peak,
                             "peak_kind": kind, "unit": "GB/s", "frac": round(ach / peak, 4),
                             "avg_launch_us": round(1e3 * d_ms / d_n, 2), "launches": d_n,
                             "traffic": stored_traffic(dom)},
                "kernel_ms": {k: [round(v[0], 3), v[2]] for k, v in kern.items()}, "clocks": clk.summary()}
        for app, idx in (("hashmin", 0), ("sssp", 1)):
            line[app] = {"ms": round(statistics.median(r[idx].elapsed_ms for r in rs), 4),
                         "modes": rs[-1][idx].mode[1:].tolist(), "policy_ms": policy_times(G, app, stream, ipg)}
    print(json.dumps(line), flush=True)


def run_config(args):
    """Secondary measured configurations (one JSON line each)."""
    import paper_2010_08781_gb300 as ipg
    import inputs
    import torch
    torch.cuda.set_device(0)
    if args.config == "c2":
        c2_line(args, max(args.steps, 5))
        return
    out = {"config": args.config}
    if args.config == "c1":  # PageRank, directed R-MAT scale 16, T = 30
        out.update(c1_summary(None, ipg))
        g = inputs.rmat_graph(16, seed=1)
        t0 = time.perf_counter()
        import oracle
        oracle.pagerank(g.n, g.row_ptr, g.col, T=30)
        dt = time.perf_counter() - t0
        out["cpu_oracle"] = {"value": round(30 * g.m / dt / 1e9, 5), "unit": "GTEPS", "cores": 1,
                             "kind": "oracle", "sample": "PageRank T=30 on the full graph", "seconds": round(dt, 2)}
        out["workload"] = "PageRank T=30 on directed R-MAT scale 16 (edge factor 16, seed 1)"
    elif args.config == "bfs_perm":
        # unit-weight SSSP (Fig. 10 exactly) with and without the early-exit pull, and what the
        # degree-class renumbering does on a graph whose vertex ids were randomly permuted
        sc = args.scale if args.scale != SCALE else C2_SCALE
        g = inputs.rmat_graph(sc, edge_factor=EDGE_FACTOR, symmetrize=True, seed=1)
        src = int(np.argmax(g.out_degree()))
        with ipg.Graph.from_inputs(g) as G:
            b = {}
            # the early exit belongs to the gather pull; the blocked pull streams every entry
            for name, kw in (("pull_early_exit", dict(policy="forced", forced_mode="pull", pr_engine="gather")),
                             ("pull_full_scan", dict(policy="forced", forced_mode="pull", pull_early_exit=0,
                                                     pr_engine="gather")),
                             ("threshold_early_exit", dict(policy="threshold", pr_engine="gather")),
                             ("threshold_full_scan", dict(policy="threshold", pull_early_exit=0, pr_engine="gather")),
                             ("pull_blocked", dict(policy="forced", forced_mode="pull", pr_engine="blocked")),
                             ("threshold_blocked", dict(policy="threshold", pr_engine="blocked"))):
                rs = [G.run("sssp", source=src, **kw) for _ in range(4)][1:]
                ms = min(r.elapsed_ms for r in rs)
                b[name] = {"ms": round(ms, 4), "gteps": round(int(rs[0].messages.sum()) / (ms * 1e-3) / 1e9, 2),
                           "supersteps": rs[0].supersteps, "modes": rs[0].mode[1:].tolist()}
        out["unit_weight_sssp"] = dict(b, workload=f"unit-weight SSSP from the largest hub on symmetrised R-MAT {sc}",
                                       edges=g.m)
        rows = {}
        for label, gg in (("ids_as_generated", c2_graph(sc)),
                          ("ids_permuted", inputs.rmat_graph(sc, edge_factor=EDGE_FACTOR, symmetrize=True, seed=1,
                                                             weighted=True, wseed=1, permute_seed=7))):
            for relabel in (False, True):
                with ipg.Graph.from_inputs(gg, relabel=relabel) as G:
                    r = {}
                    for app, kw in (("hashmin", {}), ("sssp", dict(source=0))):
                        rs = [G.run(app, policy="threshold", **kw) for _ in range(4)][1:]
                        r[app + "_ms"] = round(min(x.elapsed_ms for x in rs), 4)
                    rows[f"{label}/{'renumbered' if relabel else 'caller_order'}"] = r
        out["renumbering"] = dict(rows, workload=f"Hashmin + SSSP(0), threshold policy, symmetrised weighted R-MAT {sc}")
        out["workload"] = "unit-weight SSSP early exit; degree-class renumbering on a randomly permuted R-MAT"
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
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--scale", type=int, default=SCALE)
    ap.add_argument("--policy", default="auto")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ncu-case", default=None,
                    help="APP:MODE[:ENGINE], e.g. sssp:pull or pagerank:pull:blocked (small profiling case), or "
                         "'default': one host-driven step of the default workload (for a one-pass launch list)")
    ap.add_argument("--config", default=None, choices=["c1", "c2", "c4", "bfs_perm"],
                    help="secondary configurations: c1 PageRank scale 16, c2 Hashmin + SSSP scale 22, c4 batched, "
                         "bfs_perm unit-weight SSSP early exit and renumbering on a permuted R-MAT")
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
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+u32",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "scale": args.scale, "vertices": r["V"],
                           "edges_directed": r["Ed"], "edges_symmetrised": r["Es"], "pagerank_iterations": T_PR,
                           "pagerank_engine": "blocked pull", "hashmin_policy": args.policy,
                           "l2": "flushed between timed steps; inputs (about 13 GB) exceed L2",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "roofline": r["roofline"], "e2e": r["e2e"], "gpu_launches": r["launches"], "clocks": r["clocks"],
                "per_app": r["detail"], "memory": r["memory"]}
        if r["cpu"] is not None:
            line["cpu_baseline"] = r["cpu"]
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
