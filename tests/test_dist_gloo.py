"""The multi-rank host logic of bench.py on CPU ranks (gloo, world size 2): the max-over-ranks
step time and the whole-job unit count that the JSON line reports, the barriers around the timed
region, and the reference arm, which runs on rank 0 alone (other ranks exit at once, printing
nothing).  Every rank of the GPU arm is an independent replica (no data-path collective), so these
reductions are the only cross-rank operations."""
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


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    assert bench.dist_info() == (world, rank, rank)
    d = bench.init_dist(world, "gloo")
    assert d is dist and dist.get_world_size() == world
    # per-rank step time and unit count, as the timed region produces them
    ms = 100.0 + 10.0 * rank
    pairs = 1000 * (rank + 1)
    bench.barrier(d)
    res = {"ms_max": bench.max_over_ranks(d, ms), "pairs_all": bench.sum_over_ranks(d, pairs)}
    bench.barrier(d)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)
    dist.destroy_process_group()


def test_reductions_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        res = json.load(open(tmp_path / f"rank{r}.json"))
        assert res == {"ms_max": 110.0, "pairs_all": 3000.0}


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.init_dist(1, "gloo") is None
    assert bench.max_over_ranks(None, 3.5) == 3.5 and bench.sum_over_ranks(None, 7) == 7
    bench.barrier(None)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


@pytest.mark.slow
def test_reference_arm_line_on_rank_zero():
    env = dict(os.environ, WORLD_SIZE="2", RANK="0", LOCAL_RANK="0", MASTER_ADDR="127.0.0.1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "1", "--cpu-seconds", "4"], env=env, capture_output=True,
                       text=True, timeout=600)
    assert p.returncode == 0, p.stderr
    line = json.loads(p.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
