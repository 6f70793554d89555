"""The tensor-core contraction's pipeline stage width (M2L_OPT_TC_CHUNK: 32, 64 or 128 bytes of K
per stage) changes how operands are staged, not the MMA sequence: with whole-vector drains
(M2L_OPT_TC_DRAIN = 0) results are bit-identical. Shorter drain intervals stay within the
stated bound."""
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
        pl = lib.Plan(wl.depth, wl.p, wl.rank_tol, form="blas", precision=precision).set(tc_chunk=ch, tc_drain=0)
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



@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
def test_drain_interval_stays_within_the_stated_bound(lib, precision):
    from bounds import stated
    from gpu_util import run_gpu
    from oracle import m2l as M
    from oracle import operators as O
    wl = W.small(depth=3, p=6, density="normal", seed=11, rank_tol=1e-7)
    qs = {l: wl.multipoles(l) for l in wl.levels}
    ops = O.compressed_operators(6, 1e-7, 1.0)
    refs = {l: M.m2l_compressed(6, l, qs[l], ops, targets=np.arange(0, 8 ** l, 9))[1] for l in wl.levels}
    for drain in (0, 1, 2, 3):
        import torch
        pl = lib.Plan(3, 6, 1e-7, form="blas", precision=precision).set(tc_drain=drain, output="check")
        try:
            pl.set_stream()
            q = torch.from_numpy(wl.all_multipoles()).float().cuda()
            o = torch.empty_like(q)
            pl.apply(q, o, -1, 1)
            torch.cuda.synchronize()
            flat, off = o.double().cpu().numpy(), 0
            for l in wl.levels:
                B = wl.n_boxes(l)
                got = flat[off:off + B * pl.n].reshape(B, 1, pl.n)[np.arange(0, B, 9)]
                off += B * pl.n
                assert M.rel_l2_error(refs[l], got) < stated("blas", precision, 6), (drain, l)
        finally:
            pl.close()
