"""Sharded M2L through the CUDA library on one GPU: each slab rank's box set "own + halo" (the
partition of paper_2408_07436_gb300.shard) is applied in turn with m2l_set_boxes + m2l_apply, and
the rows each rank owns equal the unsharded result. On one GPU the ranks run one after another;
the exchange itself is tested over gloo ranks (tests/test_shard_gloo.py)."""
import numpy as np
import pytest

from paper_2408_07436_gb300 import shard
from paper_2408_07436_gb300 import workloads as W

from gpu_util import run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("form,precision", [("blas", "fp64"), ("blas", "bf16x3"), ("fft", "fp64"), ("fft", "fp32")])
@pytest.mark.parametrize("world", [2, 3])
def test_shards_through_the_library_equal_the_unsharded_level(lib, form, precision, world):
    wl = W.small(depth=4, p=4, n_rhs=2, n_points=6000, density="u11", seed=31)
    level = 4
    keys = wl.keys[level] if wl.keys[level] is not None else np.arange(8 ** level, dtype=np.uint64)
    q = wl.multipoles(level)
    rank_tol = 1e-6 if form == "blas" else 0.0
    full = run_gpu(lib, wl.depth, wl.p, {level: q}, keys={level: keys}, form=form, precision=precision,
                   output="check", level=level, R=2, rank_tol=rank_tol)[level]
    got = np.zeros_like(full)
    seen = np.zeros(len(keys), dtype=bool)
    for rank in range(world):
        own_rows, halo_rows, local_keys, own_in_local = shard.partition(keys, level, rank, world)
        local_rows = np.sort(np.concatenate([own_rows, halo_rows]))
        out = run_gpu(lib, wl.depth, wl.p, {level: q[local_rows]}, keys={level: local_keys}, form=form,
                      precision=precision, output="check", level=level, R=2, rank_tol=rank_tol)[level]
        got[own_rows] = out[own_in_local]
        assert not seen[own_rows].any()
        seen[own_rows] = True
    assert seen.all()
    if form == "blas":
        # the same sources in the same transfer-vector order for every owned target: bit for bit
        assert np.array_equal(got, full)
    else:
        # a shard's cluster occupancy can pick the other Hadamard kernel (another summation order)
        tol = 1e-14 if precision == "fp64" else 1e-6
        assert np.max(np.abs(got - full)) <= tol * np.max(np.abs(full))
