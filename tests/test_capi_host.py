"""The C-ABI library on the CPU: it loads, exports every declared symbol, validates arguments,
and its host-side plan (pseudo-inverse, SVD compression, box tables) agrees with the oracle.
No test here launches a kernel."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import geometry as G
from oracle import m2l as M
from oracle import operators as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "m2l.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(m2l_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert "m2l_plan" in names and "m2l_apply" in names and "m2l_destroy" in names
    dll = ctypes.CDLL(lib.LIB_PATH)
    for name in names:
        assert hasattr(dll, name), name


def test_peak_probe_exports_its_declared_symbol():
    import re as _re
    src = open(os.path.join(ROOT, "include", "m2l_peaks.h")).read()
    src = _re.sub(r"/\*.*?\*/", "", src, flags=_re.S)
    names = sorted(set(_re.findall(r"\b(m2l_[a-z_]+)\s*\(", src)))
    assert names == ["m2l_fma_peak"]
    from paper_2408_07436_gb300 import peaks
    dll = ctypes.CDLL(peaks.LIB_PATH)
    for name in names:
        assert hasattr(dll, name), name
    assert peaks._lib.m2l_fma_peak(0, 0, 1, None, None, None) == -1   # iters < 1: refused before any launch


def test_stated_bounds_match_the_tests_table(lib):
    from bounds import stated
    for p in range(2, 17):
        for form, precs in (("blas", ("fp64", "fp32", "tf32x3", "bf16x3")), ("fft", ("fp64", "fp32", "tf32x3"))):
            for prec in precs:
                got = lib.m2l_stated_bound(lib.FORMS[form], lib.PRECISIONS[prec], p)
                assert got == stated(form, prec, p), (form, prec, p)
    with pytest.raises(lib.M2LError):
        lib.m2l_stated_bound(lib.M2L_FORM_FFT, lib.M2L_PREC_BF16X3, 6)   # no BF16x3 FFT form
    with pytest.raises(lib.M2LError):
        lib.m2l_stated_bound(lib.M2L_FORM_BLAS, lib.M2L_PREC_FP32, 1)


def test_stage_width_option_is_validated(lib):
    h = lib.m2l_plan(3, 4, 0, 0.0)
    try:
        assert lib.m2l_set_option(h, lib.M2L_OPT_TC_CHUNK, 48) == lib.M2L_EINVAL
        for v in (0, 32, 64, 128):
            assert lib.m2l_set_option(h, lib.M2L_OPT_TC_CHUNK, v) == lib.M2L_OK
        assert lib.m2l_set_option(h, lib.M2L_OPT_TC_DRAIN, -2) == lib.M2L_EINVAL
        for v in (-1, 0, 1, 2, 64):
            assert lib.m2l_set_option(h, lib.M2L_OPT_TC_DRAIN, v) == lib.M2L_OK
        # accumulator chains of the tensor-core Hadamard: 1, 2 or 4 (0: the default)
        for v in (3, 8, -1):
            assert lib.m2l_set_option(h, lib.M2L_OPT_HADAMARD_CHAINS, v) == lib.M2L_EINVAL
        for v in (0, 1, 2, 4):
            assert lib.m2l_set_option(h, lib.M2L_OPT_HADAMARD_CHAINS, v) == lib.M2L_OK
    finally:
        lib.m2l_destroy(h)


def test_plan_rejects_bad_arguments(lib):
    for args, word in [((1, 4, 0, 0.0), "depth"), ((9, 4, 0, 0.0), "depth"), ((3, 1, 0, 0.0), "order"),
                       ((3, 4, 7, 0.0), "kernel"), ((3, 4, 0, float("nan")), "rank_tol")]:
        with pytest.raises(lib.M2LError) as e:
            lib.m2l_plan(*args)
        assert word in str(e.value)


def test_options_and_boxes_are_validated(lib):
    h = lib.m2l_plan(3, 4, 0, 0.0)
    try:
        assert lib.m2l_set_option(h, 99, 0) == lib.M2L_EINVAL
        assert lib.m2l_set_option(h, lib.M2L_OPT_FORM, 7) == lib.M2L_EINVAL
        assert lib.m2l_set_option(h, lib.M2L_OPT_PRECISION, 9) == lib.M2L_EINVAL
        assert lib.m2l_set_option(h, lib.M2L_OPT_FFT_GRID, 5) == lib.M2L_EINVAL      # < 2p - 1
        assert lib.m2l_set_option(h, lib.M2L_OPT_FFT_GRID, 7) == lib.M2L_OK
        bad = np.array([5, 3], dtype=np.uint64)
        assert lib.m2l_set_boxes(h, 2, bad.ctypes.data, 2) == lib.M2L_EINVAL         # not ascending
        big = np.array([64], dtype=np.uint64)
        assert lib.m2l_set_boxes(h, 2, big.ctypes.data, 1) == lib.M2L_EINVAL         # >= 8^level
        assert lib.m2l_set_boxes(h, 1, bad.ctypes.data, 2) == lib.M2L_EINVAL         # level < 2
        assert lib.m2l_apply(h, 1, 2, 5, 1) == lib.M2L_EINVAL                         # level > depth
        assert lib.m2l_apply(h, 1, 2, -1, 0) == lib.M2L_EINVAL                        # n_rhs < 1
    finally:
        lib.m2l_destroy(h)
    lib.m2l_destroy(None)  # NULL-safe


@pytest.mark.parametrize("level", [2, 3, 4])
def test_pair_counts_match_oracle_dense(lib, level):
    h = lib.m2l_plan(4, 4, 0, 0.0)
    try:
        assert lib.m2l_query(h, lib.M2L_Q_PAIRS, level) == M.pair_count(level)
        assert lib.m2l_query(h, lib.M2L_Q_BOXES, level) == 8 ** level
    finally:
        lib.m2l_destroy(h)


def test_pair_counts_match_oracle_sparse(lib):
    rng = np.random.default_rng(9)
    h = lib.m2l_plan(4, 4, 0, 0.0)
    try:
        for level in (2, 3, 4):
            keys = np.sort(rng.choice(8 ** level, size=max(3, 8 ** level // 5), replace=False)).astype(np.uint64)
            assert lib.m2l_set_boxes(h, level, keys.ctypes.data, len(keys)) == lib.M2L_OK
            assert lib.m2l_query(h, lib.M2L_Q_PAIRS, level) == M.pair_count(level, keys.astype(np.int64))
            assert lib.m2l_query(h, lib.M2L_Q_BOXES, level) == len(keys)
    finally:
        lib.m2l_destroy(h)


@pytest.mark.parametrize("p", [3, 4, 6])
def test_plan_pseudo_inverse_matches_oracle(lib, p):
    h = lib.m2l_plan(3, p, 0, 0.0)
    try:
        n = G.n_surface(p)
        V = lib.m2l_get_operator(h, 4)
        Ut = lib.m2l_get_operator(h, 5)
        r = lib.m2l_query(h, lib.M2L_Q_PINV_RANK)
        V = V.reshape(n, r)
        Ut = Ut.reshape(r, n)
        Vo, Uto = O.down_pinv(p, 0)          # level 0: a box of width 1, the plan's unit geometry
        assert r == Vo.shape[1]
        x = G.surface_points(p, np.zeros(3), 1.0, G.ALPHA_INNER)
        y = G.surface_points(p, np.zeros(3), 1.0, G.ALPHA_OUTER)
        K = O.laplace(x, y)
        s = np.linalg.svd(K, compute_uv=False)
        kappa = s[0] / s[r - 1]
        ref = Vo @ Uto
        assert np.linalg.norm(V @ Ut - ref) <= n * np.finfo(float).eps * kappa * np.linalg.norm(ref)
    finally:
        lib.m2l_destroy(h)


@pytest.mark.parametrize("p,tol", [(4, 1e-4), (5, 1e-6), (6, 1e-7)])
def test_plan_compression_matches_oracle(lib, p, tol):
    """Same singular values, same rank rule, same compressed operator U C_t S^T (basis free)."""
    h = lib.m2l_plan(3, p, 0, tol)
    try:
        n = G.n_surface(p)
        k = lib.m2l_query(h, lib.M2L_Q_RANK)
        s = lib.m2l_get_operator(h, 3)
        U = lib.m2l_get_operator(h, 0).reshape(n, k)
        S = lib.m2l_get_operator(h, 1).reshape(n, k)
        C = lib.m2l_get_operator(h, 2).reshape(316, k, k)
        ops = O.compressed_operators(p, tol, 1.0)
        assert k == ops["k"]
        assert np.allclose(s, ops["s_fat"], rtol=0, atol=1e-12 * s[0])
        assert np.allclose(U.T @ U, np.eye(k), atol=1e-12)
        assert np.allclose(S.T @ S, np.eye(k), atol=1e-12)
        for t in range(316):
            mine = U @ C[t] @ S.T
            ref = ops["U"] @ ops["C"][t] @ ops["S"].T
            # the plan's bases are re-orthonormalised after its Jacobi SVD; measured <= 4e-15 here
            # (3.3e-14 at p = 8, rank 1e-7)
            assert np.linalg.norm(mine - ref, 2) <= 1e-13 * np.linalg.norm(ops["K"][t], 2), t
    finally:
        lib.m2l_destroy(h)


@pytest.mark.parametrize("p,tol,dir_tol", [(5, 1e-8, 1e-5), (6, 1e-7, 1e-8)])
def test_directional_products_match_oracle(lib, p, tol, dir_tol):
    """Eq. 15 on the host: the plan's factored operator U (Ubar_t Vbar'_t^T) S^T equals the
    oracle's, which it builds from its own SVDs, to 1e-13 of ||K_t|| for every transfer vector
    (basis free: both are the rank-k_t truncation of the same compressed operator). This is the
    operator distance the FP64 directional contraction's 1e-12 parity rests on."""
    h = lib.m2l_plan(3, p, 0, tol)
    try:
        n = G.n_surface(p)
        k = lib.m2l_query(h, lib.M2L_Q_RANK)
        lib.m2l_set_option(h, lib.M2L_OPT_DIR_TOL, dir_tol)
        U = lib.m2l_get_operator(h, 0).reshape(n, k)
        S = lib.m2l_get_operator(h, 1).reshape(n, k)
        P = lib.m2l_get_operator(h, 6).reshape(316, k, k)
        ops = O.compressed_operators(p, tol, 1.0)
        d = O.directional_operators(ops["C"], dir_tol)
        for t in range(316):
            ref = ops["U"] @ (d["Ubar"][t] @ d["Vbarp"][t].T) @ ops["S"].T
            assert np.linalg.norm(U @ P[t] @ S.T - ref, 2) <= 1e-13 * np.linalg.norm(ops["K"][t], 2), t
    finally:
        lib.m2l_destroy(h)


@pytest.mark.parametrize("p,tol,dir_tol", [(5, 1e-8, 1e-5), (6, 1e-7, 1e-8)])
def test_directional_ranks_and_flops_match_oracle(lib, p, tol, dir_tol):
    """Eq. 15 on the host: the plan keeps, per transfer vector, as many singular values of C_t as
    the oracle's own SVDs (the singular values do not depend on the bases of U and S), and the
    contraction flop count is 2 k^2 per pair without the factors and 4 k k_t with them."""
    h = lib.m2l_plan(3, p, 0, tol)
    try:
        k = lib.m2l_query(h, lib.M2L_Q_RANK)
        pairs = lib.m2l_query(h, lib.M2L_Q_PAIRS, -1)
        assert lib.m2l_query(h, lib.M2L_Q_CONTRACT_FLOPS, -1) == 2 * k * k * pairs
        assert lib.m2l_query(h, lib.M2L_Q_DIR_RANK_SUM) == 0
        lib.m2l_set_option(h, lib.M2L_OPT_DIR_TOL, dir_tol)
        ops = O.compressed_operators(p, tol, 1.0)
        d = O.directional_operators(ops["C"], dir_tol)
        assert lib.m2l_query(h, lib.M2L_Q_DIR_RANK_SUM) == int(d["kt"].sum())
        # per-transfer-vector pair counts of the full levels 2..3, by brute force on the oracle's lists
        tindex = {tuple(v): i for i, v in enumerate(G.transfer_vectors())}
        flops = 0
        for level in (2, 3):
            rows, boxes, offsets, src, srow = M.interaction_csr(level)
            tgt = np.repeat(np.arange(len(rows)), np.diff(offsets))
            for v in src - boxes[rows][tgt]:
                flops += 4 * k * d["kt"][tindex[tuple(v)]]
        assert lib.m2l_query(h, lib.M2L_Q_CONTRACT_FLOPS, -1) == flops
        assert np.all(d["kt"] <= k) and d["kt"].sum() < 316 * k
    finally:
        lib.m2l_destroy(h)


@pytest.mark.parametrize("p,pc,tol", [(4, 5, 1e-6), (3, 5, 0.0), (5, 6, 1e-8)])
def test_check_order_operators_match_oracle(lib, p, pc, tol):
    """M2L_OPT_CHECK_ORDER: the plan's rectangular operators against the oracle's, basis free
    (U C_t S^T) and rank by rank, and its pseudo-inverse of the n_c x n check-to-equivalent map."""
    h = lib.m2l_plan(3, p, 0, tol)
    try:
        lib.m2l_set_option(h, lib.M2L_OPT_CHECK_ORDER, pc)
        n, nc = G.n_surface(p), G.n_surface(pc)
        assert lib.m2l_query(h, lib.M2L_Q_N) == n and lib.m2l_query(h, lib.M2L_Q_NC) == nc
        k = lib.m2l_query(h, lib.M2L_Q_RANK)
        kc = lib.m2l_query(h, lib.M2L_Q_RANK_CHECK)
        ops = O.compressed_operators(p, tol, 1.0, p_c=pc)
        assert (kc, k) == (ops["kc"], ops["k"])
        U = lib.m2l_get_operator(h, 0).reshape(nc, kc)
        S = lib.m2l_get_operator(h, 1).reshape(n, k)
        C = lib.m2l_get_operator(h, 2).reshape(316, kc, k)
        for t in (0, 99, 315):
            mine = U @ C[t] @ S.T
            ref = ops["U"] @ ops["C"][t] @ ops["S"].T
            assert np.linalg.norm(mine - ref) <= 1e-11 * np.linalg.norm(ops["K"][t])
        V = lib.m2l_get_operator(h, 4)
        Ut = lib.m2l_get_operator(h, 5)
        r = V.size // n
        V, Ut = V.reshape(n, r), Ut.reshape(r, nc)
        Vo, Uto = O.down_pinv(p, 0, p_c=pc)
        assert r == Vo.shape[1]
        x = G.surface_points(pc, np.zeros(3), 1.0, G.ALPHA_INNER)
        y = G.surface_points(p, np.zeros(3), 1.0, G.ALPHA_OUTER)
        sv = np.linalg.svd(O.laplace(x, y), compute_uv=False)
        kappa = sv[0] / sv[r - 1]
        ref = Vo @ Uto
        assert np.linalg.norm(V @ Ut - ref) <= nc * np.finfo(float).eps * kappa * np.linalg.norm(ref)
        # the option is validated: below p or above 16 is refused, 0 restores p
        assert lib.m2l_set_option(h, lib.M2L_OPT_CHECK_ORDER, p - 1) == lib.M2L_EINVAL
        assert lib.m2l_set_option(h, lib.M2L_OPT_CHECK_ORDER, 17) == lib.M2L_EINVAL
        assert lib.m2l_set_option(h, lib.M2L_OPT_CHECK_ORDER, 0) == lib.M2L_OK
        assert lib.m2l_query(h, lib.M2L_Q_NC) == n
    finally:
        lib.m2l_destroy(h)


def test_full_rank_operators_are_exact(lib):
    p = 4
    h = lib.m2l_plan(3, p, 0, 0.0)
    try:
        n = G.n_surface(p)
        assert lib.m2l_query(h, lib.M2L_Q_RANK) == n
        C = lib.m2l_get_operator(h, 2).reshape(316, n, n)
        tv = G.transfer_vectors()
        for t in (0, 100, 315):
            assert np.allclose(C[t], O.m2l_matrix(p, tv[t], 1.0), rtol=1e-14, atol=0)
    finally:
        lib.m2l_destroy(h)


def test_fft_grid_queries(lib):
    h = lib.m2l_plan(3, 6, 0, 0.0)
    try:
        assert lib.m2l_query(h, lib.M2L_Q_GRID) == 12
        assert lib.m2l_query(h, lib.M2L_Q_FREQS) == 12 * 12 * 7
        assert lib.m2l_set_option(h, lib.M2L_OPT_FFT_GRID, 11) == lib.M2L_OK
        assert lib.m2l_query(h, lib.M2L_Q_GRID) == 11
        assert lib.m2l_query(h, lib.M2L_Q_FREQS) == 11 * 11 * 6
    finally:
        lib.m2l_destroy(h)


def test_plans_alive_together_share_host_operators(lib):
    """Plans alive at the same time with the same (p, rank threshold, check order) share one
    build of the host operators: the second plan gets them at almost no setup cost, bit for bit
    equal. An option that changes one plan's operators leaves the other plan's untouched, and
    another threshold builds its own."""
    import time
    # a parameter set no other test uses, so the first build is a real one
    a = lib.m2l_plan(3, 7, 0, 3e-7)
    b = c = None
    try:
        t0 = time.perf_counter()
        ka = lib.m2l_query(a, lib.M2L_Q_RANK)
        ta = time.perf_counter() - t0
        Ca = lib.m2l_get_operator(a, 2).copy()
        b = lib.m2l_plan(4, 7, 0, 3e-7)  # another depth: the operators do not depend on the tree
        t0 = time.perf_counter()
        kb = lib.m2l_query(b, lib.M2L_Q_RANK)
        tb = time.perf_counter() - t0
        assert kb == ka
        assert np.array_equal(lib.m2l_get_operator(b, 2), Ca)
        assert np.array_equal(lib.m2l_get_operator(b, 4), lib.m2l_get_operator(a, 4))
        assert tb < 0.2 * ta, (ta, tb)
        # a check order above p rebuilds a's operators and leaves b's alone
        lib.m2l_set_option(a, lib.M2L_OPT_CHECK_ORDER, 8)
        assert lib.m2l_query(a, lib.M2L_Q_NC) == G.n_surface(8)
        assert lib.m2l_query(b, lib.M2L_Q_NC) == G.n_surface(7)
        assert lib.m2l_get_operator(a, 2).size != Ca.size or not np.array_equal(lib.m2l_get_operator(a, 2), Ca)
        assert np.array_equal(lib.m2l_get_operator(b, 2), Ca)
        # directional factors are keyed by their threshold as well
        lib.m2l_set_option(b, lib.M2L_OPT_DIR_TOL, 1e-8)
        s8 = lib.m2l_query(b, lib.M2L_Q_DIR_RANK_SUM)
        c = lib.m2l_plan(3, 7, 0, 3e-7)
        lib.m2l_set_option(c, lib.M2L_OPT_DIR_TOL, 1e-6)
        assert 0 < lib.m2l_query(c, lib.M2L_Q_DIR_RANK_SUM) < s8
        assert lib.m2l_query(c, lib.M2L_Q_RANK) == ka
    finally:
        for h in (a, b, c):
            if h is not None:
                lib.m2l_destroy(h)


def test_plans_built_from_several_threads_get_one_operator_set(lib):
    """Plans of the same parameters built concurrently (the C ABI is called without the GIL):
    whichever build publishes first, every plan ends up with the same operators."""
    import threading
    handles, ranks, errors = [None] * 6, [None] * 6, []

    def work(i):
        try:
            h = lib.m2l_plan(3, 5, 0, 1e-8)
            handles[i] = h
            ranks[i] = lib.m2l_query(h, lib.M2L_Q_RANK)
        except Exception as e:  # reported below
            errors.append(e)

    threads = [threading.Thread(target=work, args=(i,)) for i in range(6)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    try:
        assert not errors, errors
        assert len(set(ranks)) == 1
        C0 = lib.m2l_get_operator(handles[0], 2)
        for h in handles[1:]:
            assert np.array_equal(lib.m2l_get_operator(h, 2), C0)
    finally:
        for h in handles:
            if h is not None:
                lib.m2l_destroy(h)


@pytest.mark.parametrize("p,target", [(4, 1e-4), (5, 1e-6), (6, 1e-5)])
def test_rank_auto_choice_meets_the_target_in_the_oracle(lib, p, target):
    """M2L_OPT_RANK_AUTO on an explicit FP64 BLAS plan picks its rank threshold on the host (at the
    first form query); the oracle's own compressed form at that threshold, with densities of both
    signs, must then meet the target against the dense definition (Eq. 16), and a looser target
    must not give a finer rank."""
    from paper_2408_07436_gb300 import workloads as W
    pl = lib.Plan(3, p, 1e-9, form="blas", precision="fp64").set(target_tol=target, rank_auto=1)
    try:
        pl.query(lib.M2L_Q_FORM, 1)
        r = pl.current_rank_tol()
        k = pl.query(lib.M2L_Q_RANK)
    finally:
        pl.close()
    assert r == 0.0 or 1e-9 <= r <= 1e-3
    wl = W.small(depth=3, p=p, density="u11", seed=21)
    ops = O.compressed_operators(p, r, 1.0)
    assert ops["k"] == k
    for level in wl.levels:
        q = wl.multipoles(level)
        tg = np.arange(0, 8 ** level, 7)
        _, phi_c = M.m2l_compressed(p, level, q, ops, targets=tg)
        _, phi_d = M.m2l_dense(p, level, q, targets=tg)
        assert M.rel_l2_error(phi_d / 2.0 ** level, phi_c) <= target, (level, r)
    loose = lib.Plan(3, p, 1e-9, form="blas", precision="fp64").set(target_tol=target * 100, rank_auto=1)
    try:
        loose.query(lib.M2L_Q_FORM, 1)
        assert loose.current_rank_tol() >= r or r == 0.0
    finally:
        loose.close()


@pytest.mark.parametrize("p,tol", [(5, 1e-6), (6, 1e-7), (8, 1e-7)])
def test_randomised_setup_svd_matches_the_exact_truncation(lib, p, tol):
    """M2L_OPT_SVD = 1 (one-shot randomised SVD of the stacked operators, Sec. 3.1) against the
    oracle's exact compression at the same threshold: orthonormal bases, the same rank within one
    symmetry triplet (the sketch underestimates tail singular values, having no power iterations),
    and, since the threshold is relative to the largest singular value s_0 of the stacked operator,
    an error ||K_t - U U^T K_t S S^T|| below 3 tol s_0 for every t. The exact truncation, which cuts
    both sides at tol, stays below 2 tol s_0; a triplet the sketch drops at the cut has singular
    values just above tol s_0 (1.06e-7 at p = 8, tol 1e-7)."""
    n = G.n_surface(p)
    pl = lib.Plan(3, p, tol).set(svd="randomised")
    try:
        k = pl.query(lib.M2L_Q_RANK)
        U = lib.m2l_get_operator(pl.handle, 0).reshape(n, k)
        S = lib.m2l_get_operator(pl.handle, 1).reshape(n, k)
    finally:
        pl.close()
    ops = O.compressed_operators(p, tol, 1.0)
    assert abs(k - ops["k"]) <= 3
    assert np.allclose(U.T @ U, np.eye(k), atol=1e-12) and np.allclose(S.T @ S, np.eye(k), atol=1e-12)
    scale = ops["s_fat"][0]
    for t in range(0, 316, 7):
        K = ops["K"][t]
        mine = np.linalg.norm(U @ (U.T @ K @ S) @ S.T - K, 2) / scale
        exact = np.linalg.norm(ops["U"] @ ops["C"][t] @ ops["S"].T - K, 2) / scale
        assert exact < 2 * tol and mine < 3 * tol, (t, mine, exact)
