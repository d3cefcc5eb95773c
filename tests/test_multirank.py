"""The N > 1 launch path of bench.py on CPU: two gloo ranks (world size 2,
rendezvous on 127.0.0.1).  Every rank runs the same workload (replicas, weak
scaling); the timed region is the slowest rank's, which every rank receives,
and the whole-job value counts the units of all ranks.  The reference arm runs
on rank 0 only; other ranks exit 0 without work."""
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


def _rank(rank, world, port, out_dir, ms):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_max = bench.max_over_ranks(ms[rank], dist, "cpu")
    rate = bench.whole_job_rate(1000, 5, world, ms_max)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"ms_max": ms_max, "rate": rate}, f)


def test_two_gloo_ranks_take_the_slowest_rank(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    ms = [10.0, 12.5]
    mp.start_processes(_rank, args=(2, _free_port(), str(tmp_path), ms), nprocs=2, join=True,
                       start_method="spawn")
    got = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(2)]
    for g in got:
        assert g["ms_max"] == 12.5
        assert g["rate"] == pytest.approx(1000 * 5 * 2 / 0.0125)


def test_single_process_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.whole_job_rate(10, 4, 1, 2.0) == pytest.approx(20000.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
