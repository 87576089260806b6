"""The multi-GPU bookkeeping of bench.py on CPU: two replicas under a gloo
process group agree on the slowest rank's time, report whole-job throughput
from it, and draw different inputs; the reference arm runs on rank 0 only.
(The GPU path itself shards nothing: every rank runs an independent copy.)"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}",
                            rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = 10.0 + 5.0 * rank          # rank 1 is the slower replica
        slow = bench.max_over_ranks(ms, dist, "cpu")
        value = bench.job_value(1000.0, world, slow)
        seed = bench.rank_seed(1002, rank)
        out[rank] = (slow, value, seed)
    finally:
        dist.destroy_process_group()


def test_two_replicas_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0           # max over ranks
    assert res[0][1] == res[1][1] == pytest.approx(2 * 1000.0 / 0.015)
    assert res[0][2] != res[1][2]                   # independent inputs


def test_helpers_without_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_value(100.0, 1, 1000.0) == pytest.approx(100.0)


def test_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        workload = "bandlimited-N4096-T4096-E30"
        steps = 1
        warmup = 0
        cpu_sample = 8
        precision = "bf16x3"
    bench.run_reference(A())
    assert capsys.readouterr().out == ""


def test_gpus_flag_spawns_the_ranks():
    """``bench.py --gpus 2`` without a process group launches two ranks
    itself (torch.distributed.run on 127.0.0.1); on the reference arm rank 0
    alone prints the line and rank 1 exits without work."""
    import json
    import subprocess
    import sys
    env = {k: v for k, v in os.environ.items()
           if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2",
                        "--impl", "reference", "--workload", "bandlimited-N4096-T4096-E4",
                        "--steps", "1", "--warmup", "0", "--cpu-sample", "8"],
                       capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    # the step time is the measured sample time, and value is its rate
    assert line["value"] == pytest.approx(line["units_per_step"] / (line["ms_per_step"] / 1e3))


def test_gpus_flag_must_match_the_process_group():
    import subprocess
    import sys
    env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2",
                        "--impl", "reference"], capture_output=True, text=True, env=env,
                       timeout=300)
    assert r.returncode == 2 and "WORLD_SIZE" in r.stderr
