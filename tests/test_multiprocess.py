"""The multi-GPU path of bench.py is replicas only: each rank applies the same
per-GPU workload, the ranks agree on the slowest rank's time by an all-reduce
(MAX), and rank 0 reports the whole-job throughput.  Here the aggregation
runs as two gloo ranks on the CPU; the reference arm's non-zero ranks exit
without work."""
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


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        local_seconds = 1.0 + 0.5 * rank  # rank 1 is the slow one
        slowest = bench.max_over_ranks(local_seconds, ws, "cpu")
        out[rank] = (slowest, bench.job_gdofs(ws, 3_000_000, 10, slowest))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    ws, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0] == res[1]
    slowest, value = res[0]
    assert slowest == 1.5
    assert value == pytest.approx(2 * 3_000_000 * 10 / 1.5 / 1e9)


def test_single_process_is_the_identity():
    assert bench.max_over_ranks(0.25, 1, "cpu") == 0.25
    assert bench.job_gdofs(1, 1_000_000_000, 2, 2.0) == pytest.approx(1.0)


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1", MASTER_PORT="29599")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
