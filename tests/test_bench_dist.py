"""The multi-process path of bench.py on the host: world size 2 over gloo (127.0.0.1), the
barrier and the rank reductions that turn per-rank timings into the whole-job value (units of
all ranks over the slowest rank's time), and the reference arm's rank-0-only rule."""
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


def _worker(rank, world, port):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier_sync(world)
        assert bench.max_over_ranks(1.5 + rank, world) == 1.5 + world - 1
        assert bench.sum_over_ranks(rank + 1, world) == world * (world + 1) / 2
        # rank r processed (r + 1) * 100 units in (r + 1) * 10 ms: whole job = sum / slowest
        rate, ms = bench.whole_job_rate((rank + 1) * 100, (rank + 1) * 10.0, world)
        assert ms == 10.0 * world
        assert rate == pytest.approx(100 * world * (world + 1) / 2 / (ms * 1e-3))
    finally:
        dist.destroy_process_group()


def test_rank_reductions_gloo_world2():
    import torch.multiprocessing as mp
    mp.spawn(_worker, args=(2, _free_port()), nprocs=2, join=True)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.sum_over_ranks(3.0, 1) == 3.0
    assert bench.whole_job_rate(50.0, 5.0, 1) == (10000.0, 5.0)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
