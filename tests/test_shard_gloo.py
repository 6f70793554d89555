"""Sharded M2L over 2 CPU ranks (gloo): slab partition, one halo exchange per level, and the
per-rank result equal, bit for bit, to the unsharded one. The per-rank compute is the oracle
(the CPU stands in for each rank's GPU); the sharding logic is the package's."""
import os
import socket

import numpy as np
import pytest

from paper_2408_07436_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, keys, q, p, level, out_path):
    import torch.distributed as dist

    from oracle import m2l as M

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        own_rows, halo_rows, _, _ = shard.partition(keys, level, rank, world)
        local_keys, q_local, own_in_local, received = shard.exchange_halo(q[own_rows], keys, level,
                                                                         return_stats=True)
        assert received == len(halo_rows)   # exactly the halo, nothing else
        assert np.array_equal(q_local[np.searchsorted(np.sort(np.concatenate([own_rows, halo_rows])), halo_rows)],
                              q[halo_rows])
        _, phi = M.m2l_dense(p, level, q_local, keys=local_keys.astype(np.int64), targets=own_in_local)
        np.save(out_path, np.concatenate([own_rows[:, None].astype(np.float64).repeat(1, 1),
                                          phi.reshape(len(own_rows), -1)], axis=1))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_level_equals_unsharded(tmp_path, world):
    import multiprocessing as mp

    from oracle import m2l as M

    rng = np.random.default_rng(4)
    level, p = 3, 3
    keys = np.sort(rng.choice(8 ** level, size=300, replace=False)).astype(np.uint64)
    q = rng.standard_normal((len(keys), 2, 26))
    _, ref = M.m2l_dense(p, level, q, keys=keys.astype(np.int64))
    port = _free_port()
    ctx = mp.get_context("spawn")
    outs = [str(tmp_path / f"r{r}.npy") for r in range(world)]
    procs = [ctx.Process(target=_worker, args=(r, world, port, keys, q, p, level, outs[r])) for r in range(world)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    got = np.zeros_like(ref).reshape(len(keys), -1)
    seen = np.zeros(len(keys), dtype=bool)
    for path in outs:
        a = np.load(path)
        rows = a[:, 0].astype(np.int64)
        assert not seen[rows].any()
        seen[rows] = True
        got[rows] = a[:, 1:]
    assert seen.all()
    assert np.array_equal(got, ref.reshape(len(keys), -1))


def test_halo_is_within_three_planes():
    level = 4
    keys = np.arange(8 ** level, dtype=np.uint64)
    for world in (2, 4):
        for rank in range(world):
            own, halo, local, own_in = shard.partition(keys, level, rank, world)
            x0, x1 = shard.slab_bounds(level, world)[rank]
            xh = shard._x_of(keys[halo])
            assert np.all((xh >= x0 - 3) & (xh < x1 + 3))
            assert np.all((xh < x0) | (xh >= x1))
            assert np.array_equal(local[own_in], keys[own])
    # slabs tile the level exactly
    b = shard.slab_bounds(level, 3)
    assert b[0][0] == 0 and b[-1][1] == 16 and all(b[i][1] == b[i + 1][0] for i in range(2))


def test_halo_routes_cover_each_halo_once():
    """Every halo box of every rank is sent by exactly its owner, once; nothing else is sent."""
    rng = np.random.default_rng(6)
    level = 4
    keys = np.sort(rng.choice(8 ** level, size=2000, replace=False)).astype(np.uint64)
    for world in (2, 3, 5):
        routes = shard.halo_routes(keys, level, world)
        for s in range(world):
            _, halo, _, _ = shard.partition(keys, level, s, world)
            got = np.sort(np.concatenate([routes[r][s] for r in range(world)]))
            assert np.array_equal(got, np.sort(halo))
            assert len(routes[s][s]) == 0
