"""The N > 1 bench path on CPU: replicas on gloo ranks (world size 2).

The rendering path does not shard across GPUs ("replicas only"): each rank
renders the whole batch, and the job's throughput is the pixels of all ranks
over the slowest rank's time.  These tests run the host logic of that
aggregation on two gloo processes; no GPU is involved."""
import multiprocessing
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, local_ms, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank,) + bench.job_throughput(1_000_000, 5, local_ms[rank], dist))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replicas_report_all_pixels_over_the_slowest_rank():
    pytest.importorskip("torch")
    ctx = multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    local_ms = [10.0, 25.0]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, local_ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks agree: 2 ranks x 5 steps x 1 Mpix in 25 ms
    for rank, value, ms in out:
        assert ms == 25.0
        assert abs(value - 2 * 5 * 1.0 / 25e-3) < 1e-9


def test_single_process_throughput():
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.job_throughput(2_000_000, 4, 8.0)
    assert ms == 8.0 and abs(value - 2.0 * 4 / 8e-3) < 1e-9


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    assert bench.run_reference(bench.parse()) == 0
