"""The benchmark's multi-replica path on CPU: world size 2 over gloo.

bench.py runs one replica per rank with no data-path collective; ranks meet
only to take the slowest rank's time, and the whole-job rate counts every
replica's points.  Under torchrun the reference arm runs on rank 0 alone.
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


def _rank_main(rank, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=2)
    try:
        ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        slow = bench.max_over_ranks(ms, dist, "cpu")
        rate = bench.whole_job_rate(1e9, 3, slow, dist.get_world_size())
        with open(os.path.join(out, "rank%d.txt" % rank), "w") as f:
            f.write("%r %r\n" % (slow, rate))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_and_whole_job_rate(tmp_path):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(_free_port(), str(tmp_path)), nprocs=2, join=True)
    vals = [open(tmp_path / ("rank%d.txt" % r)).read().split() for r in range(2)]
    for slow, rate in vals:
        assert float(slow) == 15.0
        assert float(rate) == pytest.approx(2 * 1e9 * 3 / 0.015 / 1e9)


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.whole_job_rate(2e9, 4, 1000.0, 1) == pytest.approx(8.0)


def test_reference_arm_runs_on_rank0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, env=env, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_gradient_byte_model():
    # the compulsory bytes of a gradient shot per point and step: all passes
    # untiled, all at depth 2, and the mix the c4 timing picked in one run
    import bench
    assert bench.gradient_bytes_per_point_step(1, 1, 1) == 20 + 28 + 32
    assert bench.gradient_bytes_per_point_step(2, 2, 2) == 12 + 18 + 20
    assert bench.gradient_bytes_per_point_step(2, 1, 2) == 60
