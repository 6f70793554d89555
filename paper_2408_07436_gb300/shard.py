"""Sharding one M2L level across ranks: slab partition of the targets and the halo each rank needs.

A target tau interacts only with sources sigma at max-norm distance 2 or 3 in box indices
(transfer vectors in [-3,3]^3, Sec. 3.1). Partition the boxes of a level into slabs of
consecutive x planes, one slab per rank. A rank then needs, besides its own boxes, the
multipoles of the boxes within 3 planes on either side of its slab: one halo exchange per level
and no other communication. With the halo added, the rank applies M2L to the sparse box set
"own + halo" through the ordinary C ABI (m2l_set_boxes) and keeps the outputs of its own boxes,
which see every source they would see on a single GPU.

This module holds only the host-side bookkeeping (which boxes, which rows) and the exchange over
torch.distributed; it works with any backend (NCCL on GPUs, gloo on CPU).
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


def exchange_halo(q_level: np.ndarray, keys: np.ndarray, level: int, group=None):
    """Gather, on every rank, the multipoles of its own and halo boxes of one level.

    q_level: (B_own, R, n) multipoles of the boxes this rank owns, in Morton order.
    keys:    sorted Morton keys of ALL boxes of the level (known to every rank).
    Returns (local_keys, q_local, own_in_local) for the rank's sparse box set own + halo.
    Each rank sends its own rows; the exchange is an all-gather of variable-size blocks.
    """
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    keys = np.asarray(keys, dtype=np.uint64)
    owners = [partition(keys, level, r, world)[0] for r in range(world)]
    R, n = q_level.shape[1], q_level.shape[2]
    sizes = [len(o) for o in owners]
    mx = max(sizes) if sizes else 0
    send = torch.zeros((mx, R, n), dtype=torch.float64)
    send[: len(owners[rank])] = torch.from_numpy(np.ascontiguousarray(q_level, dtype=np.float64))
    recv = [torch.zeros_like(send) for _ in range(world)]
    dist.all_gather(recv, send, group=group)
    full = np.zeros((len(keys), R, n))
    for r in range(world):
        full[owners[r]] = recv[r][: sizes[r]].numpy()
    own_rows, halo_rows, local_keys, own_in_local = partition(keys, level, rank, world)
    local_rows = np.sort(np.concatenate([own_rows, halo_rows]))
    return local_keys, full[local_rows], own_in_local
