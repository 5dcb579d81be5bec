"""The multi-GPU path of bench.py is replicas only: every rank runs the same
step, the step time is the maximum over ranks and the throughput is the
replicas' sum.  Exercised here with two gloo ranks on the CPU; the reference
arm under a launcher prints from rank 0 only."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _rank(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(times[rank], "cpu")
        out[rank] = (ms, bench.aggregate_gflops(world, 1e9, ms))
    finally:
        torch.distributed.destroy_process_group()


def test_max_over_ranks_and_aggregate_gloo_world2():
    times = [3.0, 5.0]
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = 29600 + os.getpid() % 1000
    mp.spawn(_rank, args=(2, port, times, out), nprocs=2, join=True)
    for r in range(2):
        ms, gf = out[r]
        assert ms == 5.0
        assert gf == pytest.approx(2 * 1e9 / 5e-3 / 1e9)


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(7.5, "cpu") == 7.5
    assert bench.aggregate_gflops(1, 2e9, 2.0) == pytest.approx(1000.0)


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0
    assert p.stdout.strip() == ""
