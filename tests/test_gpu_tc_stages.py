"""The tensor-core contraction's pipeline stage width (M2L_OPT_TC_CHUNK: 32, 64 or 128 bytes of K
per stage) changes how operands are staged, not the MMA sequence: results are bit-identical."""
import numpy as np
import pytest

from paper_2408_07436_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
def test_stage_width_does_not_change_results(lib, precision):
    import torch
    wl = W.small(depth=4, p=6, n_rhs=2, n_points=3000, density="u11", rank_tol=1e-6)
    q = torch.from_numpy(wl.all_multipoles()).float().cuda()
    outs = []
    for ch in (128, 64, 32):
        pl = lib.Plan(wl.depth, wl.p, wl.rank_tol, form="blas", precision=precision).set(tc_chunk=ch)
        try:
            for l in wl.levels:
                if wl.keys[l] is not None:
                    pl.set_boxes(l, wl.keys[l])
            pl.set_stream()
            o = torch.empty_like(q)
            pl.apply(q, o, -1, wl.n_rhs)
            torch.cuda.synchronize()
            assert lib.m2l_query(pl.handle, lib.M2L_Q_DEVICE_STATUS) == 0
            outs.append(o.cpu().numpy())
        finally:
            pl.close()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    assert np.isfinite(outs[0]).all() and np.abs(outs[0]).max() > 0

