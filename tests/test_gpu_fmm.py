"""The whole FMM around the M2L plan (m2l_fmm_*): P2M, M2M, L2L, L2P and P2P on the GPU with M2L
through the library, against the oracle's own FMM (same algorithm, FP64 CPU) and against direct
summation (Eq. 16)."""
import numpy as np
import pytest

from oracle import fmm as F
from oracle import m2l as M

pytestmark = pytest.mark.gpu


def _cloud(n, seed):
    rng = np.random.default_rng(seed)
    return rng.random((n, 3)), rng.random(n)


@pytest.mark.parametrize("form", ["blas", "fft"])
def test_fmm_matches_oracle_fmm(lib, form):
    pts, q = _cloud(3000, 21)
    fmm = lib.FMM(pts, depth=3, p=4).set_m2l(form=form)
    try:
        got = fmm.evaluate(q)
    finally:
        fmm.close()
    ref = F.fmm(pts, q, 3, 4)
    assert M.rel_l2_error(ref, got) < 1e-11, form


def test_fmm_accuracy_falls_with_order_and_device_buffers(lib):
    """Against direct summation: the error falls with p (Table 6's trend); device tensors in and
    out give the same potentials as host arrays."""
    import torch
    pts, q = _cloud(20000, 22)
    direct = F.direct(pts, q)
    errs = []
    for p in (3, 5):
        fmm = lib.FMM(pts, depth=4, p=p)
        try:
            host = fmm.evaluate(q)
            dev = fmm.evaluate(torch.from_numpy(q).cuda()).cpu().numpy()
        finally:
            fmm.close()
        assert np.array_equal(host, dev)
        errs.append(M.rel_l2_error(direct, host))
    assert errs[1] < errs[0] / 10 and errs[1] < 1e-5, errs


def test_fmm_sparse_cloud_with_directional_m2l(lib):
    """Points on a sphere (most boxes empty) and the truncated, directional BLAS M2L inside."""
    rng = np.random.default_rng(23)
    v = rng.standard_normal((6000, 3))
    pts = 0.5 + 0.45 * v / np.linalg.norm(v, axis=1)[:, None]
    q = rng.standard_normal(6000)
    fmm = lib.FMM(pts, depth=4, p=5, rank_tol=1e-8).set_m2l(dir_tol=1e-9)
    try:
        got = fmm.evaluate(q)
    finally:
        fmm.close()
    assert M.rel_l2_error(F.fmm(pts, q, 4, 5), got) < 1e-6
    assert M.rel_l2_error(F.direct(pts, q), got) < 1e-4


def test_fmm_rejects_bad_arguments(lib):
    with pytest.raises(ValueError):
        lib.FMM(np.zeros((4, 2)), depth=3, p=4)
    with pytest.raises(lib.M2LError):
        lib.FMM(np.zeros((0, 3)), depth=3, p=4)
    pts, q = _cloud(500, 24)
    fmm = lib.FMM(pts, depth=2, p=3)
    try:
        assert lib._lib.m2l_fmm_set_m2l_option(fmm.handle, lib.M2L_OPT_PRECISION, lib.M2L_PREC_FP32) == lib.M2L_EINVAL
        assert lib._lib.m2l_fmm_set_m2l_option(fmm.handle, lib.M2L_OPT_CHECK_ORDER, 4) == lib.M2L_EINVAL
        assert M.rel_l2_error(F.fmm(pts, q, 2, 3), fmm.evaluate(q)) < 1e-11
    finally:
        fmm.close()
