"""GPU parity of the FFT form in TF32x3: the Hadamard products of full levels whose cluster grid
side is a multiple of 16 (levels >= 5) run on the tensor cores (tcgen05, three BF16 pieces per
operand, six products), with the spectra stored sibling-minor; the other levels take the FP32
CUDA-core kernels. Both factors of the pseudo-inverse run on the tensor cores exactly.

References: the FP64 oracle on sampled targets (check potentials, and locals through the check
potential they reproduce), the FP64 FFT form of the library on whole levels (itself held to 1e-12
of the oracle by test_gpu_parity.py), and the FP32 CUDA-core FFT form. Bound: the FFT form's
stated single-precision bound (tests/bounds.py), ten times that for the worst single target.
"""
import numpy as np
import pytest

from oracle import m2l as M
from paper_2408_07436_gb300 import workloads as W

from bounds import stated
from gpu_util import oracle_level, run_gpu

pytestmark = pytest.mark.gpu


def _sample(B, level, k, seed):
    """k targets of a full level, the first and last box of the grid among them (domain corners)."""
    rng = np.random.default_rng(seed)
    s = rng.choice(B, size=min(B, k), replace=False)
    return np.unique(np.concatenate([s, [0, B - 1]]))


@pytest.mark.parametrize("p,grid", [(4, None), (6, None), (6, 11), (8, None), (10, None)])
def test_level5_matches_oracle_sampled(lib, p, grid):
    level = 5
    wl = W.small(depth=level, p=p, density="u11", seed=40 + p)
    q = wl.multipoles(level)
    bound = stated("fft", "tf32x3", p)
    chk = run_gpu(lib, level, p, {level: q}, form="fft", precision="tf32x3", output="check", level=level,
                  fft_grid=grid)[level]
    loc = run_gpu(lib, level, p, {level: q}, form="fft", precision="tf32x3", output="locals", level=level,
                  fft_grid=grid)[level]
    tg = _sample(q.shape[0], level, 40, p)
    L_ref, phi_ref = oracle_level(p, level, q, targets=tg)
    assert M.rel_l2_error(phi_ref, chk[tg]) < bound
    assert M.max_target_rel_error(phi_ref, chk[tg]) < 10 * bound
    assert M.check_norm_error(p, level, L_ref, loc[tg]) < bound
    # the whole level against the FP32 CUDA-core kernels (another summation of the same products)
    chk32 = run_gpu(lib, level, p, {level: q}, form="fft", precision="fp32", output="check", level=level,
                    fft_grid=grid)[level]
    assert M.rel_l2_error(chk32, chk) < bound


@pytest.mark.parametrize("R", [1, 3])
def test_all_levels_and_rhs_against_fp64_fft(lib, R):
    """Depth 5 with every level: 2-4 on the CUDA cores, 5 on the tensor cores; several right-hand
    sides share the kernel matrices of a frequency. Whole levels against the FP64 FFT form."""
    wl = W.small(depth=5, p=4, n_rhs=R, density="normal", seed=51)
    qs = {l: wl.multipoles(l) for l in wl.levels}
    bound = stated("fft", "tf32x3", 4)
    got = run_gpu(lib, 5, 4, qs, form="fft", precision="tf32x3", output="check", R=R)
    ref = run_gpu(lib, 5, 4, qs, form="fft", precision="fp64", output="check", R=R)
    for l in wl.levels:
        assert M.rel_l2_error(ref[l], got[l]) < bound, l
        assert M.max_target_rel_error(ref[l], got[l]) < 10 * bound, l


@pytest.mark.parametrize("chains", [1, 2])
def test_accumulator_chains_give_the_same_products(lib, chains):
    """M2L_OPT_HADAMARD_CHAINS only splits the sums over directions into separately accumulated
    parts: every setting stays within the bound of the default one's (4) result (1: a single
    truncating chain of 26 directions, the loosest)."""
    import torch
    level, p = 5, 6
    wl = W.small(depth=level, p=p, density="normal", seed=53)
    q = wl.multipoles(level)
    outs = {}
    for ch in (0, chains):
        plan = lib.Plan(level, p, 0.0, form="fft", precision="tf32x3")
        try:
            plan.set(output="check", had_chains=ch)
            plan.set_stream()
            qd = torch.from_numpy(q.reshape(-1)).float().cuda()
            od = torch.zeros_like(qd)
            plan.apply(qd, od, level=level, n_rhs=1)
            torch.cuda.synchronize()
            assert lib.m2l_query(plan.handle, lib.M2L_Q_DEVICE_STATUS) == 0
            outs[ch] = od.cpu().double().numpy()
        finally:
            plan.close()
    assert M.rel_l2_error(outs[0], outs[chains]) < stated("fft", "tf32x3", p)


def test_accumulate_and_status(lib):
    """Locals += result, and the device status word stays clear after the tensor-core kernel."""
    import torch
    level, p = 5, 4
    wl = W.small(depth=level, p=p, density="u01", seed=52)
    q = wl.multipoles(level)
    init = {level: np.random.default_rng(3).standard_normal(q.shape)}
    base = run_gpu(lib, level, p, {level: q}, form="fft", precision="tf32x3", output="check", level=level)[level]
    acc = run_gpu(lib, level, p, {level: q}, form="fft", precision="tf32x3", output="check", level=level,
                  accumulate=True, init=init)[level]
    assert M.rel_l2_error(base + init[level], acc) < 1e-6
    plan = lib.Plan(level, p, 0.0, form="fft", precision="tf32x3")
    try:
        plan.set(output="check")
        plan.set_stream()
        qd = torch.from_numpy(q.reshape(-1)).float().cuda()
        od = torch.zeros_like(qd)
        plan.apply(qd, od, level=level, n_rhs=1)
        torch.cuda.synchronize()
        assert lib.m2l_query(plan.handle, lib.M2L_Q_DEVICE_STATUS) == 0
    finally:
        plan.close()


def test_sparse_level_takes_the_cuda_cores(lib):
    """A level with empty boxes is not full: the TF32x3 plan runs it on the FP32 kernels, still
    within the bound."""
    level, p = 5, 4
    rng = np.random.default_rng(8)
    keys = np.sort(rng.choice(8 ** level, size=9000, replace=False)).astype(np.uint64)
    q = rng.uniform(-1, 1, size=(len(keys), 1, 6 * (p - 1) ** 2 + 2))
    chk = run_gpu(lib, level, p, {level: q}, keys={level: keys}, form="fft", precision="tf32x3", output="check",
                  level=level)[level]
    tg = np.arange(0, len(keys), 300)
    _, phi_ref = oracle_level(p, level, q, keys=keys.astype(np.int64), targets=tg)
    assert M.rel_l2_error(phi_ref, chk[tg]) < stated("fft", "tf32x3", p)


def test_c3_full_size_sampled_fft_tf32x3(lib):
    """The 8M-point, depth-6, p = 8 workload (levels 5 and 6 on the tensor cores), sampled targets
    of every level against the dense definition."""
    wl = W.c3()
    qs = {l: wl.multipoles(l) for l in wl.levels}
    rng = np.random.default_rng(12)
    chk = run_gpu(lib, wl.depth, wl.p, qs, form="fft", precision="tf32x3", output="check")
    bound = stated("fft", "tf32x3", wl.p)
    for l in wl.levels:
        tg = np.sort(rng.choice(wl.n_boxes(l), size=min(wl.n_boxes(l), 24), replace=False))
        _, ref = oracle_level(wl.p, l, qs[l], targets=tg)
        assert M.rel_l2_error(ref, chk[l][tg]) < bound, l
        assert M.max_target_rel_error(ref, chk[l][tg]) < 10 * bound, l


@pytest.mark.parametrize("p", [4, 6, 8])
def test_tensor_core_pseudo_inverse_is_as_accurate_as_the_float_float_one(lib, p):
    """Below level 5 the TF32x3 FFT form differs from FP32 only in F6: both factors as exact
    products of BF16 integer slices on the tensor cores, against an FP32 GEMM for Ut_eps and the
    float-float CUDA-core sum for V_eps. Z = Ut_eps phi cancels heavily in the directions the
    check matrix damps, so the two paths' locals differ by their own rounding noise; measured in
    the check norm against the oracle, the tensor-core locals are at least as accurate (host
    emulation at p = 8: 1.40e-7 against 1.74e-7) and within the stated bound."""
    wl = W.small(depth=4, p=p, density="u11", seed=60 + p)
    qs = {l: wl.multipoles(l) for l in wl.levels}
    tc = run_gpu(lib, 4, p, qs, form="fft", precision="tf32x3", output="locals")
    ff = run_gpu(lib, 4, p, qs, form="fft", precision="fp32", output="locals")
    for l in wl.levels:
        tg = _sample(8 ** l, l, 48, l)
        L_ref, _ = oracle_level(p, l, qs[l], targets=tg)
        e_tc = M.check_norm_error(p, l, L_ref, tc[l][tg])
        e_ff = M.check_norm_error(p, l, L_ref, ff[l][tg])
        assert e_tc < stated("fft", "tf32x3", p), l
        assert e_tc <= 1.25 * e_ff + 2e-8, (l, e_tc, e_ff)
