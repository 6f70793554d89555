"""Sharding one M2L level across ranks: slab partition of the targets and the halo each rank needs.

A target tau interacts only with sources sigma at max-norm distance 2 or 3 in box indices
(transfer vectors in [-3,3]^3, Sec. 3.1). Partition the boxes of a level into slabs of
consecutive x planes, one slab per rank. A rank then needs, besides its own boxes, the
multipoles of the boxes within 3 planes on either side of its slab: one halo exchange per level
and no other communication. With the halo added, the rank applies M2L to the sparse box set
"own + halo" through the ordinary C ABI (m2l_set_boxes) and keeps the outputs of its own boxes,
which see every source they would see on a single GPU.

This module holds only the host-side bookkeeping (which boxes, which rows) and the exchange over
torch.distributed point-to-point messages; it works with any backend that has isend/irecv (gloo
on CPU, NCCL on GPUs with device tensors).
"""

from __future__ import annotations

import numpy as np

HALO = 3  # the largest |t| component (Sec. 3.1)


def _x_of(keys: np.ndarray) -> np.ndarray:
    """x box index of Morton keys (x in the lowest bit of each triple)."""
    keys = np.asarray(keys, dtype=np.uint64)
    x = np.zeros(keys.shape, dtype=np.int64)
    for b in range(21):
        x |= ((keys >> np.uint64(3 * b)) & np.uint64(1)).astype(np.int64) << b
    return x


def slab_bounds(level: int, world: int) -> list:
    """[x0, x1) plane ranges of the `world` slabs of a level (near-equal plane counts)."""
    n = 2 ** level
    cuts = [round(i * n / world) for i in range(world + 1)]
    return [(cuts[i], cuts[i + 1]) for i in range(world)]


def partition(keys: np.ndarray, level: int, rank: int, world: int):
    """Rows of `keys` (sorted Morton keys of the level's boxes) owned by `rank` and its halo rows.

    Returns (own_rows, halo_rows, local_keys, own_in_local): local_keys = keys[own ∪ halo] in
    ascending Morton order and own_in_local the positions of the owned boxes inside it.
    """
    keys = np.asarray(keys, dtype=np.uint64)
    x = _x_of(keys)
    x0, x1 = slab_bounds(level, world)[rank]
    own = (x >= x0) & (x < x1)
    need = (x >= x0 - HALO) & (x < x1 + HALO)
    halo = need & ~own
    local_rows = np.nonzero(need)[0]
    own_rows = np.nonzero(own)[0]
    halo_rows = np.nonzero(halo)[0]
    own_in_local = np.searchsorted(local_rows, own_rows)
    return own_rows, halo_rows, keys[local_rows], own_in_local


def halo_routes(keys: np.ndarray, level: int, world: int):
    """Who sends which rows to whom in one level's halo exchange.

    routes[r][s] = positions in `keys` of the boxes rank r owns that rank s needs as halo (empty
    for r == s). Every rank computes the same table from the keys alone, so no sizes are sent.
    """
    keys = np.asarray(keys, dtype=np.uint64)
    parts = [partition(keys, level, r, world) for r in range(world)]
    routes = [[np.zeros(0, dtype=np.int64) for _ in range(world)] for _ in range(world)]
    for r in range(world):
        own = parts[r][0]
        for s in range(world):
            if s != r:
                routes[r][s] = np.intersect1d(own, parts[s][1], assume_unique=True)
    return routes


def exchange_halo(q_level: np.ndarray, keys: np.ndarray, level: int, group=None, return_stats=False):
    """Fetch, by point-to-point messages, the multipoles of this rank's halo boxes of one level.

    q_level: (B_own, R, n) multipoles of the boxes this rank owns, in Morton order.
    keys:    sorted Morton keys of ALL boxes of the level (known to every rank).
    Returns (local_keys, q_local, own_in_local) for the rank's sparse box set own + halo (and, with
    return_stats, the number of rows received). Each rank sends to each other rank only the rows
    of its slab that lie within 3 planes of the other's slab, and receives exactly its halo:
    O(halo) data per rank, one exchange step per level.
    """
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    keys = np.asarray(keys, dtype=np.uint64)
    own_rows, halo_rows, local_keys, own_in_local = partition(keys, level, rank, world)
    routes = halo_routes(keys, level, world)
    q_level = np.ascontiguousarray(q_level)
    R, n = q_level.shape[1], q_level.shape[2]
    pos_in_own = {int(g): i for i, g in enumerate(own_rows)}
    reqs, recvs = [], []
    for s in range(world):
        rows = routes[rank][s]
        if s != rank and len(rows):
            buf = torch.from_numpy(np.ascontiguousarray(q_level[[pos_in_own[int(g)] for g in rows]]))
            reqs.append(dist.isend(buf, dst=s, group=group))
    for s in range(world):
        rows = routes[s][rank]
        if s != rank and len(rows):
            buf = torch.empty((len(rows), R, n), dtype=torch.from_numpy(q_level[:0]).dtype)
            reqs.append(dist.irecv(buf, src=s, group=group))
            recvs.append((rows, buf))
    for rq in reqs:
        rq.wait()
    local_rows = np.sort(np.concatenate([own_rows, halo_rows]))
    q_local = np.zeros((len(local_rows), R, n), dtype=q_level.dtype)
    q_local[own_in_local] = q_level
    received = 0
    for rows, buf in recvs:
        q_local[np.searchsorted(local_rows, rows)] = buf.numpy()
        received += len(rows)
    if return_stats:
        return local_keys, q_local, own_in_local, received
    return local_keys, q_local, own_in_local
