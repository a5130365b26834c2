"""The multi-rank logic of bench.py on CPU (two gloo ranks): the launcher's
environment, the timed region's maximum over ranks and the whole-job rate of
independent replicas; and the reference arm under a two-rank launch (rank 0
alone works and prints, rank 1 exits 0 with no output)."""
import json
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


def _rank(rank, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2",
                      RANK=str(rank), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        ws, r, local = bench.dist_setup(None)
        dist.barrier()
        elapsed = bench.timed_region_max(1.5 + rank, dist, "cpu")  # rank 1 is the slower one
        rate = bench.job_rate(1000, ws, elapsed)
        dist.barrier()
        out.put((rank, ws, r, local, elapsed, rate))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_with_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (r0, ws, r, local, elapsed, rate) in enumerate(got):
        assert (r0, ws, r, local) == (rank, 2, rank, rank)
        assert elapsed == 2.5  # the slowest rank's time, on every rank
        assert rate == 2 * 1000 / 2.5  # all ranks' units over that time


def test_single_process_is_rank_zero_of_one(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_setup(None) == (1, 0, 0)
    assert bench.timed_region_max(3.0, None, "cpu") == 3.0
    assert bench.job_rate(10, 1, 2.0) == 5.0


def test_reference_arm_under_two_ranks():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""  # rank 1 does no work and prints nothing
    env.update(RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["value"] == line["value"]
