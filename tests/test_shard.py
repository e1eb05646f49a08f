"""Within-network sharding (paper_2603_13304_gb300.shard) on CPU ranks.

Two gloo ranks split the 3 blocks of the Kagome 6 x 2 super-cell (L = 2):
each updates the outgoing messages of the blocks it owns with the FP64
oracle, the messages travel to the owners of their receivers, and the error
is all-reduced.  Two iterations reproduce the single-process oracle's
messages and errors bit for bit (the per-block arithmetic is the same and
the exchange copies bits).  Host logic only: the multi-GPU form of this
exchange is not measured on hardware (one GPU per box here).
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _setup(D=2, chi=8):
    import sys
    sys.path.insert(0, ROOT)
    import synthetic as syn
    from oracle.blockbp import BlockBP
    from oracle.geometry import Geometry
    nb = syn.kagome_neighbours(6, 2)
    t = syn.dimer_singlet_peps(nb, 2, D, seed=2, noise=1e-2, noise_seed=3)
    em = syn.initial_edge_matrices(len(nb), D, seed=7)
    geom = Geometry.kagome(6, 2, 2)
    bb = BlockBP(geom, t, chi=chi)
    bb.init_messages(em)
    return geom, bb


def test_block_owners_and_routes():
    import sys
    sys.path.insert(0, ROOT)
    from paper_2603_13304_gb300 import shard
    assert shard.block_owners(3, 2) == [0, 0, 1]
    assert shard.block_owners(5, 3) == [0, 0, 1, 1, 2]
    assert shard.block_owners(2, 4) == [0, 1]
    geom, _ = _setup()
    owners = shard.block_owners(len(geom.blocks), 2)
    r = shard.routes(geom.updates(), owners)
    assert len(r) == len(geom.updates()) == 12
    for (u, src, dst) in r:
        assert src == owners[u[0]] and dst == owners[u[2][0]]
    # block 2 (rank 1) exchanges with blocks 0 and 1 (rank 0): both directions cross ranks
    assert any(src != dst for (_, src, dst) in r)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, iters, out):
    import sys
    sys.path.insert(0, ROOT)
    from oracle.blockbp import message_distance
    from paper_2603_13304_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        geom, bb = _setup()
        owners = shard.block_owners(len(geom.blocks), world)
        held = {k: v for k, v in bb.msgs.items() if owners[k[0]] == rank}
        errs = []
        for _ in range(iters):
            e = shard.sharded_iteration(geom.updates(), owners, rank, world, held,
                                        lambda b, f: bb.update_message(b, f), message_distance)
            bb.msgs.update(held)
            errs.append(e)
        everything = [None] * world
        dist.all_gather_object(everything, held)
        if rank == 0:
            merged = {}
            for h in everything:
                merged.update(h)
            out["msgs"] = {k: [np.asarray(a) for a in v] for k, v in merged.items()}
            out["errs"] = errs
        out[f"errs{rank}"] = errs
    finally:
        dist.destroy_process_group()


def test_sharded_iterations_match_single_process():
    iters = 2
    geom, bb = _setup()
    ref_errs = [bb.step() for _ in range(iters)]
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), iters, out), nprocs=world, start_method="spawn", join=True)
    assert out["errs0"] == out["errs1"] == ref_errs
    msgs = out["msgs"]
    assert set(msgs) == set(bb.msgs)
    for k, ref in bb.msgs.items():
        assert len(msgs[k]) == len(ref)
        for a, b in zip(msgs[k], ref):
            assert a.shape == b.shape and np.array_equal(a, b), k
