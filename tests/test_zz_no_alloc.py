"""m2l_apply_noalloc: the allocation-free FP64 BLAS entry point, for callers that cannot allocate
device memory when they apply M2L (their own pool owns the memory, or a cudaMalloc's implicit
synchronisation is not acceptable in their loop). It must give m2l_apply's result, call after
call, from its static scratch array.

This file is collected last so that a run stopping at the first failure has run every other test."""
import numpy as np
import pytest

from paper_2408_07436_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the FP64 parity bound of the other GPU tests


def test_noalloc_matches_apply_on_two_calls(lib):
    import torch
    wl = W.small(depth=4, p=4, n_rhs=2, n_points=3000, density="u11")
    level = 4
    plan = lib.Plan(wl.depth, wl.p, 0.0, form="blas", precision="fp64")
    try:
        if wl.keys[level] is not None:
            plan.set_boxes(level, wl.keys[level])
        plan.set_stream()
        q = torch.from_numpy(wl.multipoles(level).reshape(-1)).cuda()
        ref = torch.empty_like(q)
        # the existing entry point: reference result, and it uploads the plan's operators
        plan.apply(q, ref, level=level, n_rhs=wl.n_rhs)
        torch.cuda.synchronize()
        ref_np = ref.cpu().numpy()
        scale = np.abs(ref_np).max()
        assert scale > 0
        out = torch.full_like(q, float("nan"))
        for call in range(2):
            out.fill_(float("nan"))
            free_before = torch.cuda.mem_get_info()[0]
            rc = lib.m2l_apply_noalloc(plan.handle, q.data_ptr(), out.data_ptr(), level, wl.n_rhs)
            assert rc == lib.M2L_OK, lib.m2l_last_error()
            torch.cuda.synchronize()
            free_after = torch.cuda.mem_get_info()[0]
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got))
            err = np.sqrt(np.sum((got - ref_np) ** 2) / np.sum(ref_np ** 2))
            assert err < TOL, (call, err)
            if call == 1:
                assert free_after == free_before  # no device memory taken by the call
    finally:
        plan.close()


def test_noalloc_rejects_oversize_and_unprepared(lib):
    import torch
    plan = lib.Plan(6, 6, 0.0, form="blas", precision="fp64")
    try:
        q = torch.zeros(8, dtype=torch.float64, device="cuda")
        o = torch.zeros(8, dtype=torch.float64, device="cuda")
        # operators not uploaded yet
        assert lib.m2l_apply_noalloc(plan.handle, q.data_ptr(), o.data_ptr(), 6, 1) == lib.M2L_EINVAL
        assert "not prepared" in lib.m2l_last_error()
        # level outside the plan
        assert lib.m2l_apply_noalloc(plan.handle, q.data_ptr(), o.data_ptr(), 7, 1) == lib.M2L_EINVAL
    finally:
        plan.close()
    # a level too large for the static scratch (262,144 boxes at p = 6) after preparation
    small = lib.Plan(6, 6, 0.0, form="blas", precision="fp64")
    try:
        small.set_stream()
        n = small.n
        q4 = torch.zeros(8 ** 2 * n, dtype=torch.float64, device="cuda")
        o4 = torch.zeros_like(q4)
        small.apply(q4, o4, level=2, n_rhs=1)
        torch.cuda.synchronize()
        big = torch.zeros(8, dtype=torch.float64, device="cuda")
        assert lib.m2l_apply_noalloc(small.handle, big.data_ptr(), big.data_ptr(), 6, 1) == lib.M2L_EINVAL
        assert "at most" in lib.m2l_last_error()
    finally:
        small.close()
