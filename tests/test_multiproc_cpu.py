"""The multi-rank host logic of bench.py on CPU ranks (gloo, world size 2).

On GB300 the ranks are independent replicas (weak scaling): every rank solves its own
problem of the same shape, and the whole-job figure is the units summed over ranks
divided by the slowest rank's time.  These tests run that aggregation over a real
process group and check the per-rank seeding and the reference arm's rank rule.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: 10 (r + 1) ms for 100 (r + 1) PCG iterations
        ms, units = bench.aggregate_over_ranks(10.0 * (rank + 1), 100 * (rank + 1), world, "cpu")
        dist.barrier()
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"ms": ms, "units": units}, f)
    finally:
        dist.destroy_process_group()


def test_aggregation_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        d = json.load(open(tmp_path / f"r{r}.json"))
        assert d["ms"] == 20.0          # the slowest rank's time
        assert d["units"] == 300.0      # units summed over ranks


def test_single_rank_aggregation_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(12.5, 7, 1, "cpu") == (12.5, 7.0)


def test_replicas_get_distinct_problems_of_one_shape():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2605_30583_gb300 import synth
    base = synth.CONFIGS["tiny"]["seed"]
    a = synth.make_config("tiny", seed=bench.replica_seed(base, 0))
    b = synth.make_config("tiny", seed=bench.replica_seed(base, 1))
    assert (a.n_cams, a.n_pts) == (b.n_cams, b.n_pts)
    assert not np.array_equal(a.pixels[:10], b.pixels[:10])
    # rank 0 is the single-GPU workload itself
    c = synth.make_config("tiny")
    assert np.array_equal(a.pixels, c.pixels)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "tiny",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "tiny",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
