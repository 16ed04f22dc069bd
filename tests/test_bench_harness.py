"""Host-side logic of the benchmark: replica aggregation over ranks (gloo,
world size 2, on the CPU), the reference arm's rank handling, and the clock
sample parser."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = [2.0, 5.0][rank]
    out[rank] = (bench.reduce_max(t, world), bench.replica_throughput(100.0, t, world))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        tmax, value = out[r]
        assert tmax == 5.0
        assert value == pytest.approx(100.0 * 2 / 5.0)


def test_reduce_max_single_rank():
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.replica_throughput(10.0, 2.0, 1) == 5.0


def test_reference_arm_other_ranks_exit_quietly(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"]) == 0
    assert capsys.readouterr().out == ""


def test_clock_summary_parsing(tmp_path):
    s = bench.ClockSampler("0")
    s.proc = object()
    s.f = open(tmp_path / "c.csv", "w+")
    s.f.write("0, 1980, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
              "0, 1965, 2070, 950.0, 0x4, Not Active, Not Active, Not Active, Active\n"
              "0, 1990, 2070, 940.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    out = s.summary()
    assert out["sm_mhz"] == 1980 and out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3


def test_summaries_are_compact_and_complete():
    """The batched and served summaries close the benchmark line: every number
    a reader needs (per-form recon/s, latencies, PSNR, speed-up) in a few
    hundred characters."""
    import json

    import bench
    leg = {"recon_per_s": 10.0, "ms": 100.0, "p50_latency_ms": 50.0, "p99_latency_ms": 99.0, "mean_psnr_db": 30.0}
    batched = {"jobs": 64, "iters_per_job": 100, "sequential": dict(leg), "batched": dict(leg),
               "batched_graph": dict(leg), "speedup_vs_sequential": 1.9,
               "policies": {name: dict(leg) for name in bench.BATCH_POLICIES},
               "tuning": {"batch_policy": bench.BATCH_POLICIES[2], "plan_adj_splits": [2, 8]}}
    b = bench.batched_summary(batched)
    assert b["policy"] == bench.BATCH_POLICIES[2]
    assert len(b["recon_per_s"]["per_policy"]) == len(bench.BATCH_POLICIES) == 3
    assert set(b["recon_per_s"]) >= {"sequential", "batched", "graph"}
    served_leg = {"recon_per_s": 1.0, "p50_latency_s": 2.0, "p99_latency_s": 3.0, "mean_psnr_db": 30.0,
                  "mean_iters": 100.0}
    served = {"requests": 16, "ranges": "128..1024^2, 90..1440 views, tol 0.0001", "sequential_capacity_per_s": 1.0,
              "loads": [{"load_vs_sequential_capacity": 1.5, "served": dict(served_leg),
                         "sequential": dict(served_leg), "speedup_recon_per_s": 1.03}]}
    v = bench.served_summary(served)
    assert v["load_1.5"]["speedup"] == 1.03 and v["ranges"].startswith("128..1024")
    assert len(json.dumps(b)) + len(json.dumps(v)) < 900
