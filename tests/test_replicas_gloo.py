"""Multi-GPU path of the benchmark, on CPU: the workloads do not shard, so N
ranks run N independent replicas with no data-path collective; the only
exchange is the max over ranks of their timings, and the whole-job value is
all ranks' units over that time.  Two gloo ranks on 127.0.0.1 check the
exchange; rank != 0 of the reference arm does no work and prints nothing."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [1.0 + rank, 10.0 * (world - rank), 5.0]
        got = bench.replica_max(local, dist, "cpu")
        out[rank] = got
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        assert out[r] == [2.0, 20.0, 5.0]


def test_whole_job_value_and_single_process_passthrough():
    # no process group: the local values come back unchanged
    assert bench.replica_max([3.0, 4.5], None, "cpu") == [3.0, 4.5]
    # 2 replicas of 1.6e9 entries each, slowest 0.02 s -> 1.6e11 entries/s
    assert bench.replica_value(2, 1.6e9, 0.02) == pytest.approx(1.6e11)
    assert bench.replica_value(1, 1.6e9, 0.02) == pytest.approx(8e10)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
