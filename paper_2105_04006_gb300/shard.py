"""Multi-GPU batch sharding (one process per GPU).

Objects are independent (Section 3.4: one periodogram per object over a
shared grid), so a batch shards across ranks with no exchange on the data
path: each rank takes a contiguous range of objects whose total cost
(sum of N_t * N_f) is as even as the boundaries allow, runs lsp_batch on its
CSR slice, and the per-object peaks are gathered on the host afterwards.
The gather is the only collective and carries 40 bytes per object.
"""
from __future__ import annotations

import numpy as np


def shard_ranges(offsets, world: int):
    """Contiguous object ranges [(o_begin, o_end)] per rank, balanced by N_t.

    Rank r takes objects whose cumulative observation count crosses the
    r-th equal share of the total; ranges are contiguous so each rank's slice
    of the CSR arrays is a view.  Empty ranges are allowed (more ranks than
    objects).
    """
    off = np.asarray(offsets, dtype=np.int64)
    n_obj = off.size - 1
    if world < 1:
        raise ValueError("world must be >= 1")
    total = int(off[-1] - off[0])
    # cost prefix at each object boundary; cut where the prefix reaches r/world
    prefix = off - off[0]
    cuts = [0]
    for r in range(1, world):
        target = total * r / world
        cut = int(np.searchsorted(prefix, target, side="left"))
        cut = min(max(cut, cuts[-1]), n_obj)
        cuts.append(cut)
    cuts.append(n_obj)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def local_slice(t, y, offsets, o_begin: int, o_end: int):
    """The CSR slice of objects [o_begin, o_end), with offsets rebased to 0."""
    off = np.asarray(offsets, dtype=np.int64)
    lo, hi = int(off[o_begin]), int(off[o_end])
    return t[lo:hi], y[lo:hi], (off[o_begin:o_end + 1] - lo).astype(np.int64)


def gather_peaks(local_peaks: np.ndarray, ranges, rank: int, per_object: int = 1, group=None):
    """Gather per-object peak records (structured numpy arrays) to rank 0.

    ``per_object`` is top_k (records per object).  Returns the global array
    in object order on rank 0 and None elsewhere.  Uses torch.distributed's
    object gather, so it works with gloo (CPU) and NCCL process groups.
    """
    import torch.distributed as dist

    world = dist.get_world_size(group)
    bufs = [None] * world if rank == 0 else None
    dist.gather_object(local_peaks, bufs, dst=0, group=group)
    if rank != 0:
        return None
    for r, (a, b) in enumerate(ranges):
        if len(bufs[r]) != (b - a) * per_object:
            raise RuntimeError(f"rank {r} returned {len(bufs[r])} records for objects [{a}, {b})")
    return np.concatenate([bufs[r] for r in range(world)])
