"""Pins of the oracle's M2L arithmetic against closed forms, invariants and brute force."""
import os

import numpy as np
import pytest

from oracle import fmm
from oracle import geometry as G
from oracle import m2l as M
from oracle import operators as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_laplace_kernel_value():
    x = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, 2.0]])
    y = np.array([[3.0, 4.0, 0.0]])
    K = O.laplace(x, y)
    assert K[0, 0] == pytest.approx(1.0 / (4 * np.pi * 5.0), rel=1e-15)
    assert K[1, 0] == pytest.approx(1.0 / (4 * np.pi * np.sqrt(4 + 4 + 4)), rel=1e-15)


def test_rel_l2_error_closed_form():
    ref = np.array([3.0, 4.0])
    approx = np.array([3.0, 4.5])
    assert M.rel_l2_error(ref, approx) == pytest.approx(0.5 / 5.0, rel=1e-15)
    assert M.rel_l2_error(ref, ref) == 0.0


def test_check_potential_matches_numpy_brute_force(rng):
    """The compiled direct sum against an explicit per-pair numpy sum (level 2, p = 3, 2 RHS)."""
    p, level = 3, 2
    n = G.n_surface(p)
    q = rng.standard_normal((64, 2, n))
    phi = M.check_potentials(p, level, q)
    w = G.box_width(level)
    boxes = G.all_boxes(level)
    for ti in (0, 5, 21, 42, 63):
        tau = boxes[ti]
        x = G.surface_points(p, G.box_centre(tau, level), w, G.ALPHA_INNER)
        ref = np.zeros((2, n))
        for si, s in enumerate(boxes):
            if np.max(np.abs(s - tau)) >= 2:  # at level 2 every far box is in I_tau
                y = G.surface_points(p, G.box_centre(s, level), w, G.ALPHA_INNER)
                for r in range(2):
                    for i in range(n):
                        for j in range(n):
                            ref[r, i] += q[si, r, j] / (4 * np.pi * np.linalg.norm(x[i] - y[j]))
        assert np.allclose(phi[ti], ref, rtol=1e-13, atol=0)


def test_pinv_moore_penrose_identities():
    """The four Penrose conditions, to the rounding a computed pseudo-inverse can reach
    (a multiple of max(M, N) * eps * cond over the kept singular values)."""
    for p in (3, 4, 5):
        x = G.surface_points(p, np.zeros(3), 1.0, G.ALPHA_INNER)
        y = G.surface_points(p, np.zeros(3), 1.0, G.ALPHA_OUTER)
        A = O.laplace(x, y)
        V, Ut = O.pinv_factors(A)
        Ap = V @ Ut
        s = np.linalg.svd(A, compute_uv=False)
        kappa = s[0] / s[V.shape[1] - 1]
        tol = 10 * max(A.shape) * np.finfo(float).eps * kappa
        nA = np.linalg.norm(A, 2)
        nAp = np.linalg.norm(Ap, 2)
        assert np.linalg.norm(A @ Ap @ A - A, 2) <= tol * nA
        assert np.linalg.norm(Ap @ A @ Ap - Ap, 2) <= tol * nAp
        assert np.linalg.norm(A @ Ap - (A @ Ap).T, 2) <= tol
        assert np.linalg.norm(Ap @ A - (Ap @ A).T, 2) <= tol


def test_pinv_threshold_rule():
    """Matrices with prescribed singular values: only those above (0 + max(M,N) eps) s0 survive (Eq. 10)."""
    rng = np.random.default_rng(11)
    m, n = 12, 9
    U, _ = np.linalg.qr(rng.standard_normal((m, m)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    eps = np.finfo(float).eps
    s = np.array([1.0, 0.5, 1e-3, 1e-8, 1e-12, 50 * m * eps, 2 * m * eps, 0.5 * m * eps, 1e-20])
    Vk, Utk = O.pinv_factors(U[:, :n] @ np.diag(s) @ V.T)
    assert Vk.shape[1] == 7 and Utk.shape[0] == 7  # 2*m*eps survives, 0.5*m*eps does not
    # a well-conditioned case: the kept part is the exact inverse, the dropped direction maps to 0
    s2 = np.array([1.0, 0.5, 0.1, 0.02, 0.01, 0.005, 0.002, 0.001, 1e-20])
    Vk, Utk = O.pinv_factors(U[:, :n] @ np.diag(s2) @ V.T)
    got = Vk @ Utk
    expect = V[:, :8] @ np.diag(1 / s2[:8]) @ U[:, :8].T
    assert np.allclose(got, expect, rtol=0, atol=1e-10)
    assert np.linalg.norm(got @ U[:, 8]) < 1e-10


def test_pinv_agrees_with_scipy():
    """Same threshold convention as SciPy's pinv (Sec. 2.1.1 says the implementation mirrors it):
    the same kept rank, and the same matrix to the rounding the conditioning allows."""
    from scipy import linalg
    for p in (3, 4, 6):
        x = G.surface_points(p, np.zeros(3), 1.0, G.ALPHA_INNER)
        y = G.surface_points(p, np.zeros(3), 1.0, G.ALPHA_OUTER)
        A = O.laplace(x, y)
        V, Ut = O.pinv_factors(A)
        ref = linalg.pinv(A)  # atol = 0, rtol = max(M, N) * eps: the rule of Eq. 10 with alpha = 0
        s = np.linalg.svd(A, compute_uv=False)
        kappa = s[0] / s[V.shape[1] - 1]
        assert V.shape[1] == np.sum(s > max(A.shape) * np.finfo(float).eps * s[0])
        assert np.linalg.norm(V @ Ut - ref) <= max(A.shape) * np.finfo(float).eps * kappa * np.linalg.norm(ref)


def test_translation_invariance_of_k():
    """K_{sigma,tau} depends only on t = idx(sigma) - idx(tau) (Sec. 2.2)."""
    p, level = 4, 4
    w = G.box_width(level)
    t = np.array([2, -3, 1])
    mats = []
    for tau in ([3, 3, 3], [5, 4, 6], [8, 9, 10]):
        tau = np.array(tau)
        x = G.surface_points(p, G.box_centre(tau, level), w, G.ALPHA_INNER)
        y = G.surface_points(p, G.box_centre(tau + t, level), w, G.ALPHA_INNER)
        mats.append(O.laplace(x, y))
    for K in mats[1:]:
        assert np.allclose(K, mats[0], rtol=1e-13, atol=0)
    # the same matrix from the operator builder (target at the origin)
    assert np.allclose(O.m2l_matrix(p, t, w), mats[0], rtol=1e-13, atol=0)


def test_shifted_root_gives_same_check_potentials(rng):
    p, level = 3, 3
    q = rng.random((8 ** level, 1, G.n_surface(p)))
    tg = np.arange(0, 512, 37)
    a = M.check_potentials(p, level, q, targets=tg)
    b = M.check_potentials(p, level, q, targets=tg, root_origin=(-3.5, 10.0, 0.25))
    assert np.allclose(a, b, rtol=1e-12, atol=0)


def test_homogeneity_across_levels(rng):
    """K scales as 1/w (degree -1, Sec. 3.1 with reading 3): check potentials double from level l to l+1
    for the same local configuration, and the locals are level independent."""
    p = 4
    n = G.n_surface(p)
    # one target with all its sources at level 3, and the same relative pattern at level 4
    tau3 = np.array([2, 3, 2])
    lst = G.interaction_list(tau3, 3)
    q = rng.random((len(lst), n))
    out = []
    for level, tau in ((3, tau3), (4, tau3 + 4)):
        w = G.box_width(level)
        x = G.surface_points(p, G.box_centre(tau, level), w, G.ALPHA_INNER)
        phi = np.zeros(n)
        for j, s in enumerate(lst):
            s = np.array(s) - tau3 + tau
            y = G.surface_points(p, G.box_centre(s, level), w, G.ALPHA_INNER)
            phi += O.laplace(x, y) @ q[j]
        L = O.pinv_apply(O.down_pinv(p, level), phi)
        out.append((phi, L))
    assert np.allclose(out[1][0], 2 * out[0][0], rtol=1e-13, atol=0)
    assert M.check_norm_error(p, 3, out[0][1][None, None], out[1][1][None, None]) < 1e-12


@pytest.mark.parametrize("p,level,g", [(3, 2, None), (4, 3, None), (4, 3, 7), (5, 3, None)])
def test_fft_m2l_equals_dense(rng, p, level, g):
    """App. A.1 is an exact reformulation of Eq. 11 (also on the alias-free 2p-1 grid)."""
    n = G.n_surface(p)
    q = rng.standard_normal((8 ** level, 2, n))
    tg = np.arange(0, 8 ** level, 29 if level == 3 else 5)
    L_d, phi_d = M.m2l_dense(p, level, q, targets=tg)
    L_f, phi_f = M.m2l_fft(p, level, q, targets=tg, g=g)
    assert M.rel_l2_error(phi_d, phi_f) < 1e-13
    assert M.check_norm_error(p, level, L_d, L_f) < 1e-12


def test_compressed_full_rank_equals_dense(rng):
    p, level = 4, 3
    n = G.n_surface(p)
    q = rng.standard_normal((8 ** level, 1, n))
    ops = O.compressed_operators(p, 0.0, G.box_width(level))
    assert ops["k"] == n
    tg = np.arange(0, 512, 11)
    L_d, phi_d = M.m2l_dense(p, level, q, targets=tg)
    L_c, phi_c = M.m2l_compressed(p, level, q, ops, targets=tg)
    assert M.rel_l2_error(phi_d, phi_c) < 1e-12
    assert M.check_norm_error(p, level, L_d, L_c) < 1e-12


def test_truncated_error_is_monotone(rng):
    p, level = 5, 3
    n = G.n_surface(p)
    q = rng.standard_normal((8 ** level, 1, n))
    tg = np.arange(0, 512, 13)
    _, phi_d = M.m2l_dense(p, level, q, targets=tg)
    errs, ks = [], []
    for tol in (1e-1, 1e-2, 1e-3, 1e-4, 1e-6, 1e-8):
        ops = O.compressed_operators(p, tol, G.box_width(level))
        _, phi_c = M.m2l_compressed(p, level, q, ops, targets=tg)
        errs.append(M.rel_l2_error(phi_d, phi_c))
        ks.append(ops["k"])
    assert all(a >= b * 0.999 for a, b in zip(errs, errs[1:])), errs
    assert all(a <= b for a, b in zip(ks, ks[1:]))
    assert errs[0] > 1e-3 and errs[-1] < 1e-7
    # the rank rule is relative to the largest singular value
    assert ks[0] < ks[-1] <= n


def _directional_spectral_errors(ops, d):
    """||C_t - Ubar_t Vbar'_t^T||_2 for every t, by an independent 2-norm evaluation."""
    return np.array([np.linalg.norm(C - Ub @ Vp.T, 2) for C, Ub, Vp in zip(ops["C"], d["Ubar"], d["Vbarp"])])


def test_directional_recompression_full_rank_is_exact(rng):
    """Eq. 15 with every singular value kept reproduces C_t, and the BLAS-M2L result with it."""
    p, level = 4, 3
    n = G.n_surface(p)
    ops = O.compressed_operators(p, 1e-6, G.box_width(level))
    d = O.directional_operators(ops["C"], 0.0)
    assert np.all(d["kt"] == ops["k"])
    scale = max(np.linalg.norm(C, 2) for C in ops["C"])
    assert _directional_spectral_errors(ops, d).max() < 1e-13 * scale
    q = rng.standard_normal((8 ** level, 2, n))
    tg = np.arange(0, 512, 17)
    _, phi_c = M.m2l_compressed(p, level, q, ops, targets=tg)
    _, phi_d = M.m2l_compressed(p, level, q, {**ops, **d}, targets=tg)
    assert M.rel_l2_error(phi_c, phi_d) < 1e-13


def test_directional_truncation_is_the_best_rank_kt_approximation():
    """Eckart-Young: the spectral-norm error of the rank-k_t truncation equals the first dropped
    singular value, which the threshold keeps below dir_tol * s_0(C_t)."""
    ops = O.compressed_operators(6, 1e-7)
    for dir_tol in (1e-3, 1e-6):
        d = O.directional_operators(ops["C"], dir_tol)
        err = _directional_spectral_errors(ops, d)
        s = d["s"]
        dropped = np.array([s[t, d["kt"][t]] if d["kt"][t] < s.shape[1] else 0.0 for t in range(len(s))])
        assert np.allclose(err, dropped, rtol=1e-6, atol=1e-14 * s[:, 0].max())
        assert np.all(err < dir_tol * s[:, 0] * (1 + 1e-9))
        assert np.all(s[np.arange(len(s)), d["kt"] - 1] >= dir_tol * s[:, 0])


def test_directional_error_is_monotone(rng):
    p, level = 5, 3
    n = G.n_surface(p)
    q = rng.standard_normal((8 ** level, 1, n))
    tg = np.arange(0, 512, 13)
    ops = O.compressed_operators(p, 1e-10, G.box_width(level))
    _, phi_ref = M.m2l_compressed(p, level, q, ops, targets=tg)
    errs, sizes = [], []
    for dir_tol in (1e-2, 1e-4, 1e-6, 1e-8):
        d = O.directional_operators(ops["C"], dir_tol)
        _, phi = M.m2l_compressed(p, level, q, {**ops, **d}, targets=tg)
        errs.append(M.rel_l2_error(phi_ref, phi))
        sizes.append(int(d["kt"].sum()))
    assert all(a >= b for a, b in zip(errs, errs[1:])), errs
    assert all(a <= b for a, b in zip(sizes, sizes[1:]))
    assert errs[0] > 1e-4 and errs[-1] < 1e-6


# Check order above the equivalent order (P_c > P_e; Sec. 5 and the optimal parameters of the
# BLAS tables): rectangular check-to-equivalent maps.

def test_check_potential_with_higher_check_order_matches_brute_force(rng):
    """n_c check points of order p + 1 against n equivalent points of order p, explicit sum."""
    p, pc, level = 3, 4, 2
    n, nc = G.n_surface(p), G.n_surface(pc)
    q = rng.standard_normal((64, 1, n))
    phi = M.check_potentials(p, level, q, p_c=pc)
    assert phi.shape == (64, 1, nc)
    w = G.box_width(level)
    boxes = G.all_boxes(level)
    for ti in (0, 27, 63):
        tau = boxes[ti]
        x = G.surface_points(pc, G.box_centre(tau, level), w, G.ALPHA_INNER)
        ref = np.zeros(nc)
        for si, s in enumerate(boxes):
            if np.max(np.abs(s - tau)) >= 2:
                y = G.surface_points(p, G.box_centre(s, level), w, G.ALPHA_INNER)
                for i in range(nc):
                    ref[i] += np.sum(q[si, 0] / (4 * np.pi * np.linalg.norm(x[i] - y, axis=1)))
        assert np.allclose(phi[ti, 0], ref, rtol=1e-13, atol=0)


def test_rectangular_pinv_penrose_identities():
    """The downward check-to-equivalent map with n_c > n rows is a least-squares problem; its
    pseudo-inverse still satisfies the four Penrose conditions to max(M,N) eps cond."""
    for p, pc in ((3, 4), (4, 6)):
        V, Ut = O.down_pinv(p, 0, p_c=pc)
        x = G.surface_points(pc, np.zeros(3), 1.0, G.ALPHA_INNER)
        y = G.surface_points(p, np.zeros(3), 1.0, G.ALPHA_OUTER)
        A = O.laplace(x, y)
        assert A.shape == (G.n_surface(pc), G.n_surface(p)) and V.shape[0] == G.n_surface(p)
        Ap = V @ Ut
        sv = np.linalg.svd(A, compute_uv=False)
        tol = 10 * max(A.shape) * np.finfo(float).eps * sv[0] / sv[V.shape[1] - 1]
        assert np.linalg.norm(A @ Ap @ A - A, 2) <= tol * np.linalg.norm(A, 2)
        assert np.linalg.norm(Ap @ A @ Ap - Ap, 2) <= tol * np.linalg.norm(Ap, 2)
        assert np.linalg.norm(A @ Ap - (A @ Ap).T, 2) <= tol
        assert np.linalg.norm(Ap @ A - (Ap @ A).T, 2) <= tol


def test_compressed_with_higher_check_order(rng):
    """With n_c > n the two bases get their own ranks (the column space of K_fat has more than n
    significant directions: its (n+1)-th singular value is still 4e-5 of the largest at p = 4,
    p_c = 5). At full rank the compressed form is exact; truncated, its error is of the order of
    the threshold."""
    p, pc, level = 4, 5, 3
    n, nc = G.n_surface(p), G.n_surface(pc)
    q = rng.standard_normal((8 ** level, 1, n))
    tg = np.arange(0, 512, 19)
    _, phi_d = M.m2l_dense(p, level, q, targets=tg, p_c=pc)
    full = O.compressed_operators(p, 0.0, G.box_width(level), p_c=pc)
    assert (full["kc"], full["k"]) == (nc, n) and full["C"].shape == (316, nc, n)
    _, phi_c = M.m2l_compressed(p, level, q, full, targets=tg, p_c=pc)
    assert M.rel_l2_error(phi_d, phi_c) < 1e-12
    assert full["s_fat"][n] / full["s_fat"][0] > 1e-5   # a k <= n check basis could not be exact
    cut = O.compressed_operators(p, 1e-6, G.box_width(level), p_c=pc)
    assert n < cut["kc"] < nc
    _, phi_t = M.m2l_compressed(p, level, q, cut, targets=tg, p_c=pc)
    assert 1e-8 < M.rel_l2_error(phi_d, phi_t) < 1e-5


def test_fmm_error_falls_with_check_order():
    """More check than equivalent points: the tiny FMM's error falls as P_c rises above P_e at
    every order tried (the effect behind the BLAS tables' P_c > P_e)."""
    rng = np.random.default_rng(1)
    pts = rng.random((800, 3))
    q = rng.random(800)
    ref = fmm.direct(pts, q)
    for p in (3, 4, 5):
        e = [M.rel_l2_error(ref, fmm.fmm(pts, q, 3, p, p_c=pc)) for pc in (p, p + 1, p + 2)]
        assert e[0] > e[1] > e[2], (p, e)


def test_symmetric_kernel_fat_and_thin_share_singular_values():
    """Sec. 3.1: for the symmetric Laplace kernel with equal surfaces one SVD suffices."""
    ops = O.compressed_operators(4, 1e-6)
    assert np.allclose(ops["s_fat"], ops["s_thin"], rtol=1e-10, atol=1e-14 * ops["s_fat"][0])


@pytest.mark.parametrize("p", [3, 5])
def test_far_field_validity(rng, p):
    """Potential inside tau from its locals vs direct from the source equivalent densities."""
    level = 3
    n = G.n_surface(p)
    q = rng.random((512, 1, n))
    ti = 300
    L, _ = M.m2l_dense(p, level, q, targets=[ti])
    tau = G.all_boxes(level)[ti]
    w = G.box_width(level)
    c = G.box_centre(tau, level)
    pts = c + (rng.random((50, 3)) - 0.5) * w
    y_loc = G.surface_points(p, c, w, G.ALPHA_OUTER)
    approx = O.laplace(pts, y_loc) @ L[0, 0]
    ref = np.zeros(50)
    for s in G.interaction_list(tau, level):
        si = int(G.morton_encode(np.array(s), level))
        y = G.surface_points(p, G.box_centre(np.array(s), level), w, G.ALPHA_INNER)
        ref += O.laplace(pts, y) @ q[si, 0]
    err = M.rel_l2_error(ref, approx)
    assert err < {3: 1e-2, 5: 1e-4}[p]


def _paper_order_error():
    rows = {}
    with open(os.path.join(GOLD, "fft_m2l_order_error.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                p, e = line.split()
                rows[int(p)] = float(e)
    return rows


def test_tiny_fmm_error_falls_with_order():
    """Whole FMM against direct summation (Eq. 16): error falls as p rises and stays within a
    factor 10 of the paper's Table 6 order of magnitude."""
    rng = np.random.default_rng(1)
    pts = rng.random((1500, 3))
    q = rng.random(1500)
    ref = fmm.direct(pts, q)
    gold = _paper_order_error()
    errs = {}
    for p in (2, 3, 4, 5, 6):
        errs[p] = M.rel_l2_error(ref, fmm.fmm(pts, q, 3, p))
    ps = sorted(errs)
    assert all(errs[a] > errs[b] for a, b in zip(ps, ps[1:])), errs
    for p, e in gold.items():
        if p in errs:
            assert errs[p] < 10 * e, (p, errs[p], e)


@pytest.mark.parametrize("p,density", [(6, "u11"), (8, "normal"), (8, "u01"), (10, "normal")])
def test_two_backward_stable_pseudo_inverses_agree_within_the_backward_bound(p, density):
    """The locals of two different backward-stable two-factor solves (LAPACK's divide-and-conquer
    SVD, which the oracle uses, and its QR-iteration SVD) agree in the check norm within
    locals_backward_bound, and that bound is not vacuous."""
    import scipy.linalg as sl
    from paper_2408_07436_gb300 import workloads as W
    wl = W.small(depth=3, p=p, density=density, seed=3)
    level = 3
    q = wl.multipoles(level)
    tg = np.arange(0, 512, 21)
    L, phi = M.m2l_dense(p, level, q, targets=tg)
    K = M.down_check_matrix(p, level)
    U, s, Vt = sl.svd(K, lapack_driver="gesvd")
    keep = s > max(K.shape) * np.finfo(np.float64).eps * s[0]
    V2, Ut2 = Vt[keep].T, (U[:, keep] / s[keep]).T
    L2 = np.einsum("ij,brj->bri", V2, np.einsum("ij,brj->bri", Ut2, phi))
    b = M.locals_backward_bound(p, level, L)
    assert M.check_norm_error(p, level, L, L2) <= b
    assert b < 1e-9


def test_explicit_pseudo_inverse_matrix_exceeds_the_backward_bound():
    """Planted: V_eps Ut_eps multiplied out into one matrix before it is applied (what the
    footnote of Sec. 2.1.1 warns against) is no backward-stable solve at p = 8, and the bound
    says so."""
    from paper_2408_07436_gb300 import workloads as W
    p, level = 8, 3
    wl = W.small(depth=3, p=p, density="u01", seed=3)
    q = wl.multipoles(level)
    tg = np.arange(0, 512, 21)
    L, phi = M.m2l_dense(p, level, q, targets=tg)
    V, Ut = O.down_pinv(p, level)
    L_bad = np.einsum("ij,brj->bri", V @ Ut, phi)
    assert M.check_norm_error(p, level, L, L_bad) > 10 * M.locals_backward_bound(p, level, L)
