"""Within-network sharding of BlockBP over ranks (one GPU per rank).

Alg. 1 updates every message of an iteration from the previous iteration's
messages, so the blocks of one network can be updated on different devices
at once (Sec. 2.2: all sides in parallel).  The partition used here:

* ownership: the blocks are split into contiguous, balanced ranges, one per
  rank; a rank keeps the incoming messages of the blocks it owns;
* update: every rank computes the outgoing messages of its own blocks from
  the incoming messages it holds (the block's own contraction needs no
  remote data);
* exchange: each outgoing message M_{a->b} goes point to point to the owner
  of the receiving block b (the owner of a, when a block neighbours itself
  through a periodic face); this is the only data exchange of an iteration;
* convergence: each rank takes the largest change over the messages it
  received, and one all-reduce (MAX) gives every rank the iteration's error.

The module holds the partition and the exchange only; the per-block compute
is the caller's (a callback), so the same driver serves any engine whose
messages are lists of tensors.  Messages travel as pickled host objects
(``torch.distributed`` object collectives), which reproduces them bit for bit.
"""
from __future__ import annotations

from typing import Callable, Dict, List, Sequence, Tuple

Key = Tuple[int, int]                 # (block, face) of the receiving side
Update = Tuple[int, int, Key]         # (sender block, its out face, receiver key)


def block_owners(n_blocks: int, world: int) -> List[int]:
    """Rank that owns each block: contiguous ranges differing by at most one."""
    if n_blocks < 0 or world < 1:
        raise ValueError("n_blocks >= 0 and world >= 1 required")
    base, extra = divmod(n_blocks, world)
    owners = []
    for r in range(world):
        owners.extend([r] * (base + (1 if r < extra else 0)))
    return owners


def routes(updates: Sequence[Update], owners: Sequence[int]) -> List[Tuple[Update, int, int]]:
    """(update, source rank, destination rank) of every message update."""
    return [(u, owners[u[0]], owners[u[2][0]]) for u in updates]


def exchange(outgoing: Dict[Key, object], owners: Sequence[int], rank: int, world: int, group=None) -> Dict[Key, object]:
    """Deliver the messages this rank produced to the owners of their
    receivers; returns the messages received for this rank's blocks (its
    own included).  One object all-to-all per iteration."""
    if world == 1:
        return dict(outgoing)
    import torch.distributed as dist
    buckets: List[Dict[Key, object]] = [dict() for _ in range(world)]
    for key, msg in outgoing.items():
        buckets[owners[key[0]]][key] = msg
    gathered: List[object] = [None] * world
    dist.all_gather_object(gathered, buckets, group=group)
    out: Dict[Key, object] = {}
    for src in range(world):
        out.update(gathered[src][rank])
    return out


def max_over_ranks(x: float, world: int, group=None) -> float:
    """The largest x over all ranks (the iteration's message error)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sharded_iteration(updates: Sequence[Update], owners: Sequence[int], rank: int, world: int,
                      held: Dict[Key, object], compute: Callable[[int, int], object],
                      distance: Callable[[object, object], float], group=None) -> float:
    """One synchronous iteration on this rank.

    held: the incoming messages of the blocks this rank owns (replaced in
    place by the new ones); compute(block, face): the outgoing message of
    that update, from the messages held before the iteration; distance(old,
    new): the change of one message.  Returns the largest change over all
    ranks."""
    outgoing = {}
    for (blk, face, recv) in updates:
        if owners[blk] == rank:
            outgoing[recv] = compute(blk, face)
    received = exchange(outgoing, owners, rank, world, group)
    err = 0.0
    for key, msg in received.items():
        if key in held:
            err = max(err, distance(held[key], msg))
    held.update(received)
    return max_over_ranks(err, world, group)
