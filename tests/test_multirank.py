"""The multi-rank (replicas) path of bench.py on the CPU: two gloo ranks.

The suggestion path does not shard: each rank holds a whole replica of the
database and answers its own queries, so the only cross-rank steps are the
barrier around the timed region and the max over ranks of the elapsed time.
These tests run those steps with world size 2 on the gloo backend, and the
reference arm under torchrun, where rank 0 alone prints the JSON line.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as tdist
    import bench
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.setup_dist() == (world, rank, rank)
        # each rank's elapsed time differs; all must see the slowest
        mine = 1.5 + rank
        slowest = bench.max_over_ranks(mine, torch.device("cpu"), world)
        tdist.barrier()
        rate = bench.whole_job_rate(1000.0, 4, slowest, world)
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"slowest": slowest, "rate": rate}, f)
    finally:
        tdist.destroy_process_group()


def test_max_over_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    for r in res:
        assert r["slowest"] == 2.5
        # 2 ranks x 1,000 units x 4 steps in 2.5 s
        assert r["rate"] == pytest.approx(3200.0)


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, None, 1) == 3.25
    assert bench.whole_job_rate(10.0, 3, 2.0, 1) == 15.0


def test_reference_arm_under_torchrun(tmp_path):
    env = dict(os.environ)
    env.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--workload", "tiny_k3", "--steps", "2", "--warmup", "3", "--ref-sample", "4"]
    p = subprocess.run(cmd, cwd=str(tmp_path), env=env, capture_output=True, text=True,
                       timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 2
    assert d["value"] > 0 and d["e2e"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle"


def test_captured_traffic_only_for_the_captured_run():
    """The bench attaches an ncu-captured DRAM figure only to a run that
    matches the capture: the whole workload, the cosine and the plan tuning
    the capture was taken under."""
    sys.path.insert(0, ROOT)
    import bench
    got = bench.captured_traffic("scan_bf16", "precision", "bf16", "cosine", None, True)
    assert got is not None and got > 0
    # a cut of the workload, another metric or a tuned plan: no figure
    assert bench.captured_traffic("scan_bf16", "precision", "bf16", "cosine", None, False) is None
    assert bench.captured_traffic("scan_bf16", "precision", "bf16", "euclidean", None, True) is None
    assert bench.captured_traffic("scan_bf16", "precision", "bf16", "cosine",
                                  {"list_len": 4}, True) is None
    # the batch was captured under its autotuned plan: only that plan matches
    tuned = {"items_per_block": 1, "list_len": 16, "l2_share_pct": 0}
    assert bench.captured_traffic("scan_bf16", "batching", "bf16", "cosine", tuned, True) > 0
    assert bench.captured_traffic("scan_bf16", "batching", "bf16", "cosine", None, True) is None
    assert bench.captured_traffic("scan_bf16", "batching", "bf16", "cosine",
                                  {"items_per_block": 4, "list_len": 16}, True) is None
    # never captured
    assert bench.captured_traffic("scan_fp8", "precision", "fp8", "cosine", None, True) is None


def test_oracle_sample_is_bounded():
    """The CPU baseline's sample stays within its bounds whatever the
    workload's size."""
    sys.path.insert(0, ROOT)
    import bench
    import fsgen
    w = fsgen.make("tiny_k3")
    n = bench.oracle_sample_size(w, 15.0, 8, 1024)
    assert 1 <= n <= w.q
    # a huge per-query cost still takes the lower bound, capped by the queries
    big = fsgen.Workload("x", 0, 10**9, 256, 50, [3])
    assert bench.oracle_sample_size(big, 15.0, 8, 1024) == 8
