"""The N > 1 path of the benchmark on CPU: independent replicas, one
max-reduction of the timing over ranks (gloo, world size 2)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        secs = [0.75, 1.25][rank]
        m = bench.max_over_ranks(secs, world)
        # whole-job throughput: all ranks' units over the slowest rank's time
        units = 12 * 3
        out[rank] = (m, world * units / m)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    assert out[0] == out[1]
    assert out[0][0] == pytest.approx(1.25)
    assert out[0][1] == pytest.approx(2 * 36 / 1.25)


def test_single_rank_is_identity():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.max_over_ranks(0.5, 1) == 0.5
