"""Host logic of the N-rank bench on CPU: two gloo ranks, each with its own timed
region; the job time is the slower rank's and the throughput counts every rank's
units (replicas, weak scaling).  No GPU and no data-path collective are involved."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 1.5 + rank  # seconds of this rank's timed region
        t = bench.max_over_ranks(mine, dist, torch.device("cpu"))
        v = bench.job_throughput(200000, 10, world, t)
        torch.save({"t": t, "v": v}, os.path.join(out, f"r{rank}.pt"))
    finally:
        dist.destroy_process_group()


def test_two_rank_timing(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    if not torch.distributed.is_available():
        pytest.skip("torch.distributed not built")
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [torch.load(os.path.join(tmp_path, f"r{r}.pt")) for r in range(world)]
    for r in res:
        assert r["t"] == 2.5  # the slower rank's time on every rank
        assert r["v"] == pytest.approx(200000 * 10 * 2 / 2.5)


def test_single_process_passthrough():
    import bench
    assert bench.max_over_ranks(3.25, None, None) == 3.25
    assert bench.job_throughput(100, 4, 1, 2.0) == 200.0
