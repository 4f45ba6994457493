"""bench.py's multi-GPU path is replicas only: each rank runs its own workload and
the whole-job rate is (messages of all ranks) / (slowest rank's time). The host
logic is checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, m = bench.reduce_over_ranks(10.0 + 5 * rank, 1000 * (rank + 1), world, "cpu")
    out.put((rank, t, m))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_reduction_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, t, m in res:
        assert t == 15.0 and m == 3000.0  # slowest rank's time, all ranks' messages


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_over_ranks(7.5, 42, 1) == (7.5, 42.0)


def test_reference_arm_prints_one_line(capsys, monkeypatch):
    """--impl reference times the CPU oracle; a tiny scale keeps this a unit test."""
    import sys
    import json
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                                      "--scale", "10"])
    bench.main()
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["e2e"]["h2d_bytes_per_step"] == 0


def test_clock_summary_keeps_the_timed_region(tmp_path):
    """The clock record of a bench line comes from the samples taken inside the timed
    region; throttle reasons active there are reported, those outside are not."""
    import time as _time
    from datetime import datetime

    import bench

    def line(t, mhz, hw="Not Active"):
        ts = datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return f"{ts}, 0, {mhz}, 2070, 900.5, 0x0, {hw}, Not Active, Not Active, Not Active\n"

    c = bench.ClockSampler(0)
    c.proc = object()  # sampling "ran"
    t0 = _time.time()
    with open(c.path, "w") as f:
        f.write(line(t0 - 1.0, 1000, "Active"))  # before the region: ignored
        f.write(line(t0 + 0.10, 2070))
        f.write(line(t0 + 0.20, 2055))
        f.write(line(t0 + 0.30, 2070))
        f.write(line(t0 + 2.0, 900, "Active"))  # after the region: ignored
    c.t0, c.t1 = t0, t0 + 0.35
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070 and s["reasons"] == []
    assert s["window"] == "timed region"

    c = bench.ClockSampler(0)
    c.proc = object()
    with open(c.path, "w") as f:
        f.write(line(t0 - 1.0, 1000))
        f.write(line(t0 + 0.5, 2040, "Active"))
    c.t0, c.t1 = t0, t0 + 0.01  # shorter than the sampling interval
    s = c.summary()
    assert s["samples"] == 1 and s["sm_mhz"] == 2040 and s["reasons"] == ["hw_slowdown"]
    assert s["window"].startswith("nearest")


def test_kernel_count_of_a_run():
    """gpu_launches counts the library's kernels per run from the modes it ran:
    PageRank, 30 blocked pulls: k_pr_init + selector, then scatter + accumulate +
    selector per superstep; Hashmin: two superstep-0 kernels + selector, a blocked
    pull = scatter + accumulate + apply + selector, a gather pull or a dense push =
    3, a sparse push = compaction + push + apply + selector."""
    import bench
    assert bench.launches_of([0] + [2] * 30, "pagerank", blocked=True) == 2 + 30 * 3
    assert bench.launches_of([0] + [2] * 30, "pagerank") == 2 + 30 * 2
    modes = [0, 2, 2, 2, 1, 0, 0]
    assert bench.launches_of(modes, "hashmin", blocked=True) == 3 + 3 * 4 + 3 + 4 + 4
    assert bench.launches_of(modes, "hashmin") == 3 + 3 * 3 + 3 + 4 + 4
