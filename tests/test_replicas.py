"""The replicas path of bench.py on CPU: two gloo ranks stand in for two GPUs.

The path does not shard (each solve is one chain of dependent steps), so N
GPUs run N independent replicas: disjoint x0 seeds, no collective in the data
path, and one all-reduce of the per-rank times after the timed region.  These
tests run that host logic with world_size 2 over gloo; the reference arm's
rank rule (rank 0 alone works and prints) is checked by launching bench.py as
rank 1, and its JSON line (the CPU oracle on a bounded sample) against the
headline's metric, unit and config.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        K = 7
        # a slow rank 1: its total (and its e2e total) must decide the job's rate
        local = [100.0 + 50.0 * rank, 120.0 + 10.0 * rank]
        mx = bench.max_over_ranks(local)
        seeds = bench.replica_seeds(rank, 3 + K)
        every = [None] * world
        dist.all_gather_object(every, seeds)
        q.put((rank, mx, bench.whole_job_rate(world, K, mx[0]), every))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank_and_disjoint_seeds():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, rate, every in out:
        assert mx == [150.0, 130.0]                     # max over ranks, element by element
        assert rate == pytest.approx(2 * 7 / 0.150)     # all ranks' solves over the slowest time
        assert len(set(every[0]) & set(every[1])) == 0  # no x0 solved twice
        assert all(len(set(s)) == len(s) for s in every)


def test_max_over_ranks_without_a_process_group_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 1.5]) == [3.0, 1.5]
    assert bench.whole_job_rate(1, 20, 400.0) == pytest.approx(50.0)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_line_keeps_the_contract():
    """The reference arm (the CPU oracle on a bounded sample) prints one JSON
    line with the headline's metric, unit and config, so the two arms'
    lines compare like for like."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "LOCAL_RANK", "WORLD_SIZE")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "solves/s"
    assert d["config"] == bench.config_dict(1, "fp32")
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"] == {"value": d["value"], "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
