"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element.

Check potentials are compared with Eq. 16 directly. Locals are compared through the check
potential they reproduce (oracle.m2l.check_norm_error): the pseudo-inverse amplifies rounding
by up to cond(K_tau) (1e5 at p = 4, 1e9 at p = 6), and the FMM only ever uses the locals
through potentials they generate (the footnote of Sec. 2.1.1).

Tolerances: FP64 paths 1e-12 (the benchmark spec's bound) on check potentials, truncated and
directional forms included: the plan's compressed and directional operators equal the oracle's
own to 1e-13 of ||K_t|| (tests/test_capi_host.py), so they add at most a few 1e-14. FP64 locals:
1e-12, or the backward-error bound of the pseudo-inverse solve where that is larger
(oracle.m2l.locals_backward_bound: two correct backward-stable solves differ by that much in the
check norm at p >= 8, where cond(K_tau) reaches 1e12). FP32 paths: the relative rounding of a
sum of 189 n products in single precision, bounded by 5e-6 on check potentials.

Per target: every full-size test also bounds the largest relative error of a single target box
(oracle.m2l.max_target_rel_error), since one wrong box among many barely moves the level-wide
Eq. 16: 1e-11 in FP64, ten times the level-wide bound in single precision.
"""
import numpy as np
import pytest

from oracle import m2l as M
from oracle import operators as O
from oracle import geometry as G
from paper_2408_07436_gb300 import workloads as W

from bounds import stated
from gpu_util import levels_of, oracle_level, run_gpu

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 5e-6
FP64_TARGET_TOL = 1e-11


def locals_tol(p, level, L_ref):
    """FP64 bound on locals in the check norm: 1e-12, or the pseudo-inverse's backward bound."""
    return max(FP64_TOL, M.locals_backward_bound(p, level, L_ref))


def _qs(wl, dtype=np.float64):
    return {l: wl.multipoles(l) for l in wl.levels}


@pytest.mark.parametrize("form", ["blas", "fft"])
def test_c1_fp64_all_levels(lib, form):
    wl = W.c1()
    qs = _qs(wl)
    chk = run_gpu(lib, wl.depth, wl.p, qs, form=form, output="check")
    loc = run_gpu(lib, wl.depth, wl.p, qs, form=form, output="locals")
    for l in wl.levels:
        L_ref, phi_ref = oracle_level(wl.p, l, qs[l])
        assert M.rel_l2_error(phi_ref, chk[l]) < FP64_TOL, (form, l)
        assert M.check_norm_error(wl.p, l, L_ref, loc[l]) < FP64_TOL, (form, l)


@pytest.mark.parametrize("form", ["blas", "fft"])
def test_fp64_high_order(lib, form):
    """p = 8 in FP64: check potentials to rounding; locals within the spread the pseudo-inverse
    threshold itself allows. Singular values within rounding of (max(M, N) eps) s_0 (Eq. 10) are
    kept by one SVD and dropped by another, and for p >= 8 that moves the locals by a few 1e-12
    in the check norm (measured 4.3e-12), whatever the arithmetic."""
    wl = W.small(depth=3, p=8, density="normal", seed=3)
    qs = _qs(wl)
    chk = run_gpu(lib, 3, 8, qs, form=form, output="check")
    loc = run_gpu(lib, 3, 8, qs, form=form, output="locals")
    for l in wl.levels:
        tg = np.arange(0, 8 ** l, max(1, 8 ** l // 24))
        L_ref, phi_ref = oracle_level(8, l, qs[l], targets=tg)
        assert M.rel_l2_error(phi_ref, chk[l][tg]) < FP64_TOL, (form, l)
        assert M.check_norm_error(8, l, L_ref, loc[l][tg]) < locals_tol(8, l, L_ref), (form, l)


def test_fft_odd_grid_equals_dense(lib):
    wl = W.small(depth=3, p=4)
    qs = _qs(wl)
    chk = run_gpu(lib, 3, 4, qs, form="fft", output="check", fft_grid=7)
    for l in wl.levels:
        _, phi_ref = oracle_level(4, l, qs[l])
        assert M.rel_l2_error(phi_ref, chk[l]) < FP64_TOL


@pytest.mark.parametrize("p", [2, 3, 5])
def test_other_orders_fp64(lib, p):
    wl = W.small(depth=3, p=p, density="normal")
    qs = _qs(wl)
    for form in ("blas", "fft"):
        chk = run_gpu(lib, 3, p, qs, form=form, output="check")
        for l in wl.levels:
            _, phi_ref = oracle_level(p, l, qs[l])
            assert M.rel_l2_error(phi_ref, chk[l]) < FP64_TOL, (form, p, l)


def test_truncated_blas_matches_compressed_oracle(lib):
    p, tol, depth = 6, 1e-7, 3
    wl = W.small(depth=depth, p=p, density="u11", rank_tol=tol)
    qs = _qs(wl)
    chk = run_gpu(lib, depth, p, qs, rank_tol=tol, output="check")
    ops = O.compressed_operators(p, tol, 1.0)
    for l in wl.levels:
        _, phi_c = M.m2l_compressed(p, l, qs[l], ops)   # unit-width operators: unit check potential
        assert M.rel_l2_error(phi_c, chk[l]) < FP64_TOL
        assert M.max_target_rel_error(phi_c, chk[l]) < FP64_TARGET_TOL
        _, phi_d = oracle_level(p, l, qs[l])
        assert M.rel_l2_error(phi_d, chk[l]) < 1e-6      # the truncation itself


@pytest.mark.parametrize("form", ["blas", "fft"])
@pytest.mark.parametrize("R", [1, 3])
def test_sparse_boxes_and_multiple_rhs(lib, form, R):
    wl = W.small(depth=4, p=4, n_rhs=R, n_points=400, density="normal")
    assert wl.is_sparse()
    qs = _qs(wl)
    keys = {l: wl.keys[l] for l in wl.levels}
    chk = run_gpu(lib, wl.depth, wl.p, qs, keys=keys, form=form, output="check", R=R)
    loc = run_gpu(lib, wl.depth, wl.p, qs, keys=keys, form=form, output="locals", R=R)
    for l in wl.levels:
        k = None if keys[l] is None else keys[l].astype(np.int64)
        L_ref, phi_ref = oracle_level(wl.p, l, qs[l], keys=k)
        assert M.rel_l2_error(phi_ref, chk[l]) < FP64_TOL, (form, l)
        assert M.check_norm_error(wl.p, l, L_ref, loc[l]) < FP64_TOL, (form, l)


@pytest.mark.parametrize("form", ["blas", "fft"])
def test_single_level_and_accumulate(lib, form):
    wl = W.small(depth=3, p=3, n_rhs=2)
    qs = _qs(wl)
    allv = run_gpu(lib, 3, 3, qs, form=form, R=2)
    one = run_gpu(lib, 3, 3, {3: qs[3]}, form=form, level=3, R=2)
    assert np.allclose(one[3], allv[3], rtol=0, atol=1e-13 * np.abs(allv[3]).max())
    init = {l: np.ones_like(qs[l]) for l in wl.levels}
    acc = run_gpu(lib, 3, 3, qs, form=form, R=2, accumulate=True, init=init)
    for l in wl.levels:
        assert np.allclose(acc[l], allv[l] + 1.0, rtol=1e-12, atol=1e-12 * np.abs(allv[l]).max())


def test_host_buffers_equal_device_buffers(lib):
    wl = W.small(depth=3, p=4)
    qs = _qs(wl)
    a = run_gpu(lib, 3, 4, qs)
    b = run_gpu(lib, 3, 4, qs, host=True)
    for l in wl.levels:
        assert np.array_equal(a[l], b[l])


@pytest.mark.parametrize("form", ["blas", "fft"])
def test_fp32_forms(lib, form):
    wl = W.small(depth=3, p=4, density="u11")
    qs = _qs(wl)
    chk = run_gpu(lib, 3, 4, qs, form=form, precision="fp32", output="check")
    for l in wl.levels:
        _, phi_ref = oracle_level(4, l, qs[l])
        assert M.rel_l2_error(phi_ref, chk[l]) < FP32_TOL, (form, l)


def test_edge_cases(lib):
    # depth 2: one level, every pair in the box's far field interacts
    wl = W.small(depth=2, p=3)
    qs = _qs(wl)
    for form in ("blas", "fft"):
        chk = run_gpu(lib, 2, 3, qs, form=form, output="check")
        _, phi_ref = oracle_level(3, 2, qs[2])
        assert M.rel_l2_error(phi_ref, chk[2]) < FP64_TOL
    # a single non-empty box at every level: no interactions, zero output
    keys = {2: np.array([5], dtype=np.uint64), 3: np.array([40], dtype=np.uint64)}
    qs1 = {2: np.ones((1, 1, G.n_surface(3))), 3: np.ones((1, 1, G.n_surface(3)))}
    for form in ("blas", "fft"):
        out = run_gpu(lib, 3, 3, qs1, keys=keys, form=form)
        assert np.all(out[2] == 0) and np.all(out[3] == 0)
    # two far boxes only: each sees exactly the other
    keys = {2: np.array([0, 63], dtype=np.uint64)}
    q2 = {2: np.random.default_rng(4).random((2, 1, G.n_surface(3)))}
    for form in ("blas", "fft"):
        chk = run_gpu(lib, 2, 3, q2, keys=keys, form=form, output="check")
        _, phi_ref = oracle_level(3, 2, q2[2], keys=keys[2].astype(np.int64))
        assert M.rel_l2_error(phi_ref, chk[2]) < FP64_TOL


def test_error_codes(lib):
    import torch
    h = lib.m2l_plan(3, 4, 0, 0.0)
    try:
        q = torch.zeros(584 * 56, dtype=torch.float32, device="cuda")
        o = torch.zeros_like(q)
        lib.m2l_set_option(h, lib.M2L_OPT_FORM, lib.M2L_FORM_FFT)
        lib.m2l_set_option(h, lib.M2L_OPT_PRECISION, lib.M2L_PREC_BF16X3)   # no BF16x3 FFT form
        assert lib.m2l_apply(h, q.data_ptr(), o.data_ptr(), -1, 1) == lib.M2L_EUNSUPPORTED
        lib.m2l_set_option(h, lib.M2L_OPT_PRECISION, lib.M2L_PREC_FP32)
        assert lib.m2l_apply(h, q.data_ptr(), q.data_ptr() + 64, -1, 1) == lib.M2L_EINVAL   # overlap
        assert "overlap" in lib.m2l_last_error()
    finally:
        lib.m2l_destroy(h)


@pytest.mark.parametrize("form,precision", [("blas", "fp64"), ("fft", "fp64"), ("blas", "fp32"), ("fft", "fp32")])
def test_c2_full_size_sampled(lib, form, precision):
    """The 1M-point, depth-5, p = 6 workload at full size, sampled targets checked one by one."""
    wl = W.c2()
    qs = _qs(wl)
    tol = wl.rank_tol if form == "blas" else 0.0
    grid = wl.fft_grid if form == "fft" else None  # (2p-1)^3 grid for this workload
    chk = run_gpu(lib, wl.depth, wl.p, qs, rank_tol=tol, form=form, precision=precision, output="check",
                  fft_grid=grid)
    bound = FP64_TOL if precision == "fp64" else FP32_TOL
    ops = O.compressed_operators(wl.p, tol, 1.0) if form == "blas" else None
    rng = np.random.default_rng(5)
    for l in wl.levels:
        B = wl.n_boxes(l)
        sample = np.sort(rng.choice(B, size=min(B, 48), replace=False))
        if form == "blas":
            _, phi_ref = M.m2l_compressed(wl.p, l, qs[l], ops, targets=sample)
        else:
            _, phi_ref = oracle_level(wl.p, l, qs[l], targets=sample)
        assert M.rel_l2_error(phi_ref, chk[l][sample]) < bound, (l,)
        tbound = FP64_TARGET_TOL if precision == "fp64" else 10 * bound
        assert M.max_target_rel_error(phi_ref, chk[l][sample]) < tbound, (l,)


# Directional recompression (Eq. 15). Where the plan and the oracle keep the same k_t (checked on
# the host, test_capi_host), the rank-k_t truncation of C_t is unique, so the two agree to
# rounding although their SVD bases differ.
def _directional_ref(p, level, q, rank_tol, dir_tol, keys=None, targets=None):
    ops = O.compressed_operators(p, rank_tol, 1.0)
    d = O.directional_operators(ops["C"], dir_tol)
    return M.m2l_compressed(p, level, q, {**ops, **d}, keys=keys, targets=targets)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_directional_contraction_matches_oracle(lib, precision):
    wl = W.small(depth=3, p=5, density="u11", rank_tol=1e-8)
    qs = _qs(wl)
    chk = run_gpu(lib, 3, 5, qs, rank_tol=1e-8, precision=precision, output="check", dir_tol=1e-5)
    for l in wl.levels:
        L_ref, phi_ref = _directional_ref(5, l, qs[l], 1e-8, 1e-5)
        e = M.rel_l2_error(phi_ref, chk[l])
        assert e < (FP64_TOL if precision == "fp64" else FP32_TOL), (precision, l, e)
        # and the factorisation stays close to the unfactored operators (about 10 dir_tol)
        _, phi_dense = oracle_level(5, l, qs[l])
        assert M.rel_l2_error(phi_dense, chk[l]) < 1e-3


def test_directional_sparse_multi_rhs(lib):
    wl = W.small(depth=4, p=4, n_rhs=3, n_points=500, density="normal", rank_tol=1e-6)
    qs = _qs(wl)
    keys = {l: wl.keys[l] for l in wl.levels}
    chk = run_gpu(lib, wl.depth, wl.p, qs, keys=keys, rank_tol=1e-6, output="check", R=3, dir_tol=1e-4)
    loc = run_gpu(lib, wl.depth, wl.p, qs, keys=keys, rank_tol=1e-6, output="locals", R=3, dir_tol=1e-4)
    for l in wl.levels:
        k = None if keys[l] is None else keys[l].astype(np.int64)
        L_ref, phi_ref = _directional_ref(wl.p, l, qs[l], 1e-6, 1e-4, keys=k)
        assert M.rel_l2_error(phi_ref, chk[l]) < FP64_TOL, l
        # locals through the unit-width pseudo-inverse of the oracle's check potentials
        L_ref = M.locals_from_check(wl.p, 0, phi_ref)
        assert M.check_norm_error(wl.p, 0, L_ref, loc[l]) < locals_tol(wl.p, 0, L_ref), l


def test_c2_full_size_sampled_directional(lib):
    """The 1M-point workload's FP64 BLAS configuration with the directional factors at 1e-8."""
    wl = W.c2()
    qs = _qs(wl)
    chk = run_gpu(lib, wl.depth, wl.p, qs, rank_tol=wl.rank_tol, output="check", dir_tol=wl.rank_tol / 10)
    rng = np.random.default_rng(8)
    for l in wl.levels:
        B = wl.n_boxes(l)
        sample = np.sort(rng.choice(B, size=min(B, 32), replace=False))
        _, phi_ref = _directional_ref(wl.p, l, qs[l], wl.rank_tol, wl.rank_tol / 10, targets=sample)
        assert M.rel_l2_error(phi_ref, chk[l][sample]) < FP64_TOL, l
        assert M.max_target_rel_error(phi_ref, chk[l][sample]) < FP64_TARGET_TOL, l
        _, phi_dense = oracle_level(wl.p, l, qs[l], targets=sample)
        assert M.rel_l2_error(phi_dense, chk[l][sample]) < 2e-6, l


# Check order above the equivalent order (M2L_OPT_CHECK_ORDER; the BLAS tables' P_c > P_e).
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_check_order_full_rank_matches_dense(lib, precision):
    wl = W.small(depth=3, p=4, density="u11")
    qs = _qs(wl)
    chk = run_gpu(lib, 3, 4, qs, precision=precision, output="check", check_order=5)
    loc = run_gpu(lib, 3, 4, qs, precision=precision, output="locals", check_order=5)
    tol = FP64_TOL if precision == "fp64" else FP32_TOL
    for l in wl.levels:
        L_ref, phi_ref = M.m2l_dense(4, l, qs[l], p_c=5)
        assert chk[l].shape[2] == G.n_surface(5)
        assert M.rel_l2_error(phi_ref / 2.0 ** l, chk[l]) < tol, (precision, l)
        assert M.check_norm_error(4, l, L_ref, loc[l], p_c=5) < tol, (precision, l)


def test_check_order_truncated_directional_sparse(lib):
    wl = W.small(depth=4, p=5, n_rhs=3, n_points=500, density="normal", rank_tol=1e-8)
    qs = _qs(wl)
    keys = {l: wl.keys[l] for l in wl.levels}
    kw = dict(keys=keys, rank_tol=1e-8, R=3, check_order=6, dir_tol=1e-5)
    chk = run_gpu(lib, wl.depth, wl.p, qs, output="check", **kw)
    loc = run_gpu(lib, wl.depth, wl.p, qs, output="locals", **kw)
    ops = O.compressed_operators(5, 1e-8, 1.0, p_c=6)
    d = O.directional_operators(ops["C"], 1e-5)
    for l in wl.levels:
        k = None if keys[l] is None else keys[l].astype(np.int64)
        _, phi_ref = M.m2l_compressed(5, l, qs[l], {**ops, **d}, keys=k, p_c=6)
        assert M.rel_l2_error(phi_ref, chk[l]) < FP64_TOL, l
        L_ref = M.locals_from_check(5, 0, phi_ref, p_c=6)
        assert M.check_norm_error(5, 0, L_ref, loc[l], p_c=6) < max(
            FP64_TOL, M.locals_backward_bound(5, 0, L_ref, p_c=6)), l
        _, phi_dense = M.m2l_dense(5, l, qs[l], keys=k, p_c=6)
        assert M.rel_l2_error(phi_dense / 2.0 ** l, chk[l]) < 1e-3, l


def test_check_order_refuses_fft_and_tensor_cores(lib):
    wl = W.small(depth=2, p=4)
    qs = _qs(wl)
    for form, precision in (("fft", "fp64"), ("blas", "tf32x3"), ("blas", "bf16x3")):
        with pytest.raises(lib.M2LError) as e:
            run_gpu(lib, 2, 4, qs, form=form, precision=precision, check_order=5)
        assert e.value.code == lib.M2L_EUNSUPPORTED, (form, precision)


# Split tensor-core precisions (tcgen05): bounds on check potentials. TF32x3 pieces carry 22
# mantissa bits, so the result sits near FP32 rounding (measured 5.2e-7 to 1.4e-6 for p = 4..10);
# BF16x3 pieces carry about 17 (measured up to 5.9e-6, largest for densities of both signs).
TC_TOL = {"tf32x3": 3e-6, "bf16x3": 1.2e-5}   # the stated bounds for p >= 6 (tests/bounds.py)


def _status(lib, handle):
    return lib.m2l_query(handle, lib.M2L_Q_DEVICE_STATUS)


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
def test_tensor_core_forms_small(lib, precision):
    wl = W.small(depth=3, p=4, density="u11")
    qs = _qs(wl)
    chk = run_gpu(lib, 3, 4, qs, precision=precision, output="check")
    loc = run_gpu(lib, 3, 4, qs, precision=precision, output="locals")
    for l in wl.levels:
        L_ref, phi_ref = oracle_level(4, l, qs[l])
        e = M.rel_l2_error(phi_ref, chk[l])
        assert e < stated("blas", precision, 4), (precision, l, e)
        assert M.check_norm_error(4, l, L_ref, loc[l]) < stated("blas", precision, 4)


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
def test_tensor_core_sparse_multi_rhs_truncated(lib, precision):
    wl = W.small(depth=4, p=5, n_rhs=3, n_points=500, density="normal", rank_tol=1e-6)
    qs = _qs(wl)
    keys = {l: wl.keys[l] for l in wl.levels}
    chk = run_gpu(lib, wl.depth, wl.p, qs, keys=keys, rank_tol=1e-6, precision=precision, output="check", R=3)
    ops = O.compressed_operators(wl.p, 1e-6, 1.0)
    for l in wl.levels:
        k = None if keys[l] is None else keys[l].astype(np.int64)
        _, phi_c = M.m2l_compressed(wl.p, l, qs[l], ops, keys=k)
        e = M.rel_l2_error(phi_c, chk[l])
        assert e < TC_TOL[precision], (precision, l, e)


def test_watchdog_expiry_is_reported_and_the_context_survives(lib):
    """A bounded wait that nothing completes (the self-test barrier) runs out, is reported as
    M2L_ETIMEOUT with its site code, is cleared by the query, and the CUDA context keeps working:
    the tensor-core contraction afterwards still matches the oracle."""
    import ctypes

    import torch
    wl = W.small(depth=3, p=4, density="u11")
    qs = _qs(wl)
    plan = lib.Plan(3, 4, 0.0, form="blas", precision="tf32x3")
    try:
        plan.set_stream()
        lib.m2l_selftest_watchdog(plan.handle, 1000)
        out = ctypes.c_longlong(0)
        rc = lib._lib.m2l_query(plan.handle, lib.M2L_Q_DEVICE_STATUS, -1, ctypes.byref(out))
        assert rc == lib.M2L_ETIMEOUT and out.value == lib.M2L_WAIT_SELFTEST
        assert "ran out" in lib.m2l_last_error()
        assert _status(lib, plan.handle) == 0          # cleared by the query above
        with pytest.raises(lib.M2LError):
            lib.m2l_selftest_watchdog(plan.handle, 0)  # bad argument, nothing launched
        q = torch.from_numpy(wl.all_multipoles()).float().cuda()
        o = torch.empty_like(q)
        plan.set(output="check")
        plan.apply(q, o, -1, 1)
        assert _status(lib, plan.handle) == 0
        flat = o.double().cpu().numpy()
        off = 0
        for l in wl.levels:
            B = wl.n_boxes(l)
            got = flat[off:off + B * plan.n].reshape(B, 1, plan.n)
            off += B * plan.n
            _, phi_ref = oracle_level(4, l, qs[l])
            assert M.rel_l2_error(phi_ref, got) < TC_TOL["tf32x3"], l
    finally:
        plan.close()


def test_tensor_core_status_clear(lib):
    import torch
    wl = W.small(depth=3, p=4)
    plan = lib.Plan(3, 4, 0.0, form="blas", precision="tf32x3")
    try:
        plan.set_stream()
        q = torch.from_numpy(wl.all_multipoles()).float().cuda()
        o = torch.empty_like(q)
        plan.apply(q, o, -1, 1)
        assert _status(lib, plan.handle) == 0
        assert torch.isfinite(o).all()
    finally:
        plan.close()


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
def test_c2_full_size_sampled_tensor_cores(lib, precision):
    wl = W.c2()
    qs = _qs(wl)
    chk = run_gpu(lib, wl.depth, wl.p, qs, rank_tol=wl.rank_tol, precision=precision, output="check")
    ops = O.compressed_operators(wl.p, wl.rank_tol, 1.0)
    rng = np.random.default_rng(6)
    for l in wl.levels:
        B = wl.n_boxes(l)
        sample = np.sort(rng.choice(B, size=min(B, 48), replace=False))
        _, phi_ref = M.m2l_compressed(wl.p, l, qs[l], ops, targets=sample)
        assert M.rel_l2_error(phi_ref, chk[l][sample]) < TC_TOL[precision], (precision, l)
        assert M.max_target_rel_error(phi_ref, chk[l][sample]) < 10 * TC_TOL[precision], (precision, l)


# Stated bounds of the single-precision paths per order p (tests/bounds.py; the library's autotuner
# uses the same table): check potentials and locals in the check norm. The tensor-core forms need
# k_pad <= 256, so at p >= 8 they run at rank 1e-7 and are compared with the oracle's compressed
# form at that rank (the truncation itself is not theirs).
@pytest.mark.parametrize("p", [4, 6, 8, 10])
def test_single_precision_bounds_over_orders(lib, p):
    wl = W.small(depth=3, p=p, density="normal", seed=11)
    qs = _qs(wl)
    refs, crefs = {}, {}
    ops = O.compressed_operators(p, 1e-7, 1.0) if p > 6 else None
    for l in wl.levels:
        tg = np.arange(0, 8 ** l, max(1, 8 ** l // 24))
        L, phi = M.m2l_dense(p, l, qs[l], targets=tg)
        refs[l] = (tg, L, phi / 2.0 ** l)
        if ops is not None:
            _, phic = M.m2l_compressed(p, l, qs[l], ops, targets=tg)
            crefs[l] = (tg, M.locals_from_check(p, 0, phic), phic)
    for form, prec in (("blas", "fp32"), ("fft", "fp32"), ("blas", "tf32x3"), ("blas", "bf16x3")):
        bound = stated(form, prec, p)
        tc = prec in ("tf32x3", "bf16x3")
        rank = 1e-7 if (tc and p > 6) else 0.0
        chk = run_gpu(lib, 3, p, qs, rank_tol=rank, form=form, precision=prec, output="check")
        loc = run_gpu(lib, 3, p, qs, rank_tol=rank, form=form, precision=prec, output="locals")
        for l in wl.levels:
            if rank > 0:
                tg, L_ref, phi_ref = crefs[l]
                lev = 0   # unit-width operators
            else:
                tg, L_ref, phi_ref = refs[l]
                lev = l
            assert M.rel_l2_error(phi_ref, chk[l][tg]) < bound, (form, prec, p, l)
            assert M.max_target_rel_error(phi_ref, chk[l][tg]) < 10 * bound, (form, prec, p, l)
            assert M.check_norm_error(p, lev, L_ref, loc[l][tg]) < bound, (form, prec, p, l)


def test_c3_full_size_sampled(lib):
    """The 8M-point, depth-6, p = 8 workload at full size, sampled targets checked one by one:
    BF16x3 against the oracle's compressed form, the FP64 BLAS form with the directional factors
    against the oracle's directional form and the dense definition, and FP64 FFT against the
    dense definition."""
    wl = W.c3()
    qs = _qs(wl)
    rng = np.random.default_rng(9)
    samples = {l: np.sort(rng.choice(wl.n_boxes(l), size=min(wl.n_boxes(l), 24), replace=False)) for l in wl.levels}
    dense = {l: oracle_level(wl.p, l, qs[l], targets=samples[l])[1] for l in wl.levels}
    ops = O.compressed_operators(wl.p, wl.rank_tol, 1.0)
    chk = run_gpu(lib, wl.depth, wl.p, qs, rank_tol=wl.rank_tol, precision="bf16x3", output="check")
    for l in wl.levels:
        _, ref = M.m2l_compressed(wl.p, l, qs[l], ops, targets=samples[l])
        assert M.rel_l2_error(ref, chk[l][samples[l]]) < TC_TOL["bf16x3"], ("bf16x3", l)
        assert M.max_target_rel_error(ref, chk[l][samples[l]]) < 10 * TC_TOL["bf16x3"], ("bf16x3", l)
    chk = run_gpu(lib, wl.depth, wl.p, qs, rank_tol=wl.rank_tol, output="check", dir_tol=wl.dir_tol)
    d = O.directional_operators(ops["C"], wl.dir_tol)
    for l in wl.levels:
        _, ref = M.m2l_compressed(wl.p, l, qs[l], {**ops, **d}, targets=samples[l])
        assert M.rel_l2_error(ref, chk[l][samples[l]]) < FP64_TOL, ("fp64 directional", l)
        assert M.max_target_rel_error(ref, chk[l][samples[l]]) < FP64_TARGET_TOL, ("fp64 directional", l)
        # the truncation at 1e-7 and the directional cut at 1e-8 against the dense definition
        assert M.rel_l2_error(dense[l], chk[l][samples[l]]) < 2e-8, ("fp64 directional vs dense", l)
    chk = run_gpu(lib, wl.depth, wl.p, qs, form="fft", output="check")
    for l in wl.levels:
        assert M.rel_l2_error(dense[l], chk[l][samples[l]]) < FP64_TOL, ("fft fp64", l)
        assert M.max_target_rel_error(dense[l], chk[l][samples[l]]) < FP64_TARGET_TOL, ("fft fp64", l)


def test_c4_full_size_sampled(lib):
    """The sphere-surface workload (2M points, depth 6, p = 6, 32 right-hand sides, empty boxes
    pruned) at full size, sampled targets checked one by one: the split tensor-core forms against
    the oracle's compressed form and FP32 FFT against the dense definition."""
    wl = W.c4()
    qs = _qs(wl)
    keys = {l: wl.keys[l] for l in wl.levels}
    okeys = {l: None if keys[l] is None else keys[l].astype(np.int64) for l in wl.levels}
    rng = np.random.default_rng(10)
    samples = {l: np.sort(rng.choice(wl.n_boxes(l), size=min(wl.n_boxes(l), 16), replace=False)) for l in wl.levels}
    ops = O.compressed_operators(wl.p, wl.rank_tol, 1.0)
    for prec in ("bf16x3", "tf32x3"):
        chk = run_gpu(lib, wl.depth, wl.p, qs, keys=keys, rank_tol=wl.rank_tol, precision=prec, output="check",
                      R=wl.n_rhs)
        for l in wl.levels:
            _, ref = M.m2l_compressed(wl.p, l, qs[l], ops, keys=okeys[l], targets=samples[l])
            assert M.rel_l2_error(ref, chk[l][samples[l]]) < TC_TOL[prec], (prec, l)
            assert M.max_target_rel_error(ref, chk[l][samples[l]]) < 10 * TC_TOL[prec], (prec, l)
    chk = run_gpu(lib, wl.depth, wl.p, qs, keys=keys, form="fft", precision="fp32", output="check", R=wl.n_rhs)
    for l in wl.levels:
        _, ref = oracle_level(wl.p, l, qs[l], keys=okeys[l], targets=samples[l])
        assert M.rel_l2_error(ref, chk[l][samples[l]]) < stated("fft", "fp32", wl.p), ("fft fp32", l)
        assert M.max_target_rel_error(ref, chk[l][samples[l]]) < 10 * stated("fft", "fp32", wl.p), ("fft fp32", l)
