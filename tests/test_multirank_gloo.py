"""The multi-rank harness on CPU: two gloo ranks exercise the pieces
bench.py uses under torchrun -- per-rank problem seeds (independent problems,
no data-path collective), the batched workload's shards (every instance on
exactly one rank), the barrier, the maximum of the ranks' elapsed times, the
sum of their work and the whole-job rate -- and the reference arm's rank
rule (rank 0 alone prints; other ranks exit 0 without work)."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out_dir: str):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    from paper_2601_07508_b300 import inputs
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    p = inputs.largest_prime_below_pow2(40)
    A, B = inputs.problem(40 + bench.rank_seed(rank), 8, 8, 8, p)
    dist.barrier()
    # the batched workload: each rank's shard of the 512 instances
    shard = bench.batch_shard(512, rank, world)
    everyone = [None] * world
    dist.all_gather_object(everyone, shard)
    work = bench.sum_over_ranks(float(len(shard)), dist, "cpu")
    elapsed = 1.5 + rank  # this rank's "time"
    slowest = bench.max_over_ranks(elapsed, dist, "cpu")
    rate = bench.job_rate(2.0 * 8 ** 3, 3, world, slowest)
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"slowest": slowest, "rate": rate, "a00": int(A[0, 0]), "sum": int(A.sum() % p),
                   "shards": everyone, "work": work}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_share_timing_but_not_data(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r0 = json.loads((tmp_path / "rank0.json").read_text())
    r1 = json.loads((tmp_path / "rank1.json").read_text())
    assert r0["slowest"] == r1["slowest"] == 2.5  # the job's time is the slowest rank's
    assert r0["rate"] == r1["rate"] == pytest.approx(2.0 * 8 ** 3 * 3 * 2 / 2.5 / 1e9)
    assert (r0["a00"], r0["sum"]) != (r1["a00"], r1["sum"])  # independent problems per rank
    # the batched workload's shards cover every instance exactly once
    s0, s1 = r0["shards"]
    assert r1["shards"] == r0["shards"] and sorted(s0 + s1) == list(range(512)) and not set(s0) & set(s1)
    assert r0["work"] == r1["work"] == 512.0


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--size", "64",
                        "--steps", "1", "--warmup", "0", "--bits", "20"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env["RANK"], env["LOCAL_RANK"] = "0", "0"
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--size", "64",
                        "--steps", "1", "--warmup", "0", "--bits", "20", "--cpu-seconds", "1"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0

