"""Planted mistakes: each plausible bug, planted in the oracle on the CPU, must fail a pin."""
import numpy as np
import pytest

from oracle import fmm
from oracle import geometry as G
from oracle import m2l as M
from oracle import operators as O


def _fmm_error(p=4):
    rng = np.random.default_rng(1)
    pts = rng.random((600, 3))
    q = rng.random(600)
    return M.rel_l2_error(fmm.direct(pts, q), fmm.fmm(pts, q, 3, p))


def test_reference_fmm_error_is_small():
    assert _fmm_error() < 1e-3


def test_source_on_wrong_surface_is_caught(monkeypatch):
    """M2L source taken on the outer (upward check) radius instead of its equivalent surface."""
    def bad(p, width, p_c=None):
        return (G.surface_points(p, np.zeros(3), width, G.ALPHA_INNER),
                G.surface_points(p, np.zeros(3), width, G.ALPHA_OUTER))
    monkeypatch.setattr(M, "m2l_surfaces", bad)
    assert not _fmm_error() < 1e-3  # NaN (coincident points) fails the pin as well


def test_wrong_check_radius_is_caught(monkeypatch):
    """Target check points moved off the inner radius."""
    def bad(p, width, p_c=None):
        return (G.surface_points(p, np.zeros(3), width, 1.5),
                G.surface_points(p, np.zeros(3), width, G.ALPHA_INNER))
    monkeypatch.setattr(M, "m2l_surfaces", bad)
    assert not _fmm_error() < 1e-3  # NaN (coincident points) fails the pin as well


def test_adjacent_sources_in_list_are_caught(monkeypatch):
    monkeypatch.setattr(G, "is_adjacent_or_same", lambda a, b: bool(np.all(np.asarray(a) == np.asarray(b))))
    sizes = [len(G.interaction_list(tau, 3)) for tau in G.all_boxes(3)[::17]]
    assert max(sizes) != 189


def test_flipped_transfer_vector_is_caught(rng, monkeypatch):
    p, level = 3, 3
    q = rng.standard_normal((512, 1, G.n_surface(p)))
    tg = np.arange(0, 512, 31)
    _, phi_d = M.m2l_dense(p, level, q, targets=tg)
    orig = O.m2l_matrix
    monkeypatch.setattr(O, "m2l_matrix", lambda p, t, width=1.0, p_c=None: orig(p, -np.asarray(t), width, p_c))
    ops = O.compressed_operators(p, 0.0, G.box_width(level))
    _, phi_c = M.m2l_compressed(p, level, q, ops, targets=tg)
    assert M.rel_l2_error(phi_d, phi_c) > 1e-6


def test_transposed_operator_is_caught(rng, monkeypatch):
    p, level = 3, 3
    q = rng.standard_normal((512, 1, G.n_surface(p)))
    tg = np.arange(0, 512, 31)
    _, phi_d = M.m2l_dense(p, level, q, targets=tg)
    orig = O.m2l_matrix
    monkeypatch.setattr(O, "m2l_matrix", lambda p, t, width=1.0, p_c=None: orig(p, t, width, p_c).T)
    ops = O.compressed_operators(p, 0.0, G.box_width(level))
    _, phi_c = M.m2l_compressed(p, level, q, ops, targets=tg)
    assert M.rel_l2_error(phi_d, phi_c) > 1e-6


def test_shifted_kernel_grid_is_caught(rng, monkeypatch):
    p, level = 3, 2
    q = rng.standard_normal((64, 1, G.n_surface(p)))
    tg = np.arange(0, 64, 9)
    _, phi_d = M.m2l_dense(p, level, q, targets=tg)
    orig = O.kernel_grid
    monkeypatch.setattr(O, "kernel_grid", lambda p, t, width=1.0, g=None: np.roll(orig(p, t, width, g), 1, axis=2))
    _, phi_f = M.m2l_fft(p, level, q, targets=tg)
    assert M.rel_l2_error(phi_d, phi_f) > 1e-6


def test_dropped_term_in_direct_sum_is_caught(rng, monkeypatch):
    """Drop the last source of every list: the brute-force pin disagrees."""
    p, level = 3, 2
    q = rng.standard_normal((64, 1, G.n_surface(p)))
    good = M.check_potentials(p, level, q, targets=[0])
    orig = G.interaction_lists_vectorised

    def bad(targets, level, source_slot=None):
        off, src, rows = orig(targets, level, source_slot)
        keep = np.ones(len(rows), bool)
        keep[off[1:] - 1] = False
        new_off = off - np.arange(len(off))
        return new_off, src[keep], rows[keep]
    monkeypatch.setattr(G, "interaction_lists_vectorised", bad)
    assert M.rel_l2_error(good, M.check_potentials(p, level, q, targets=[0])) > 1e-6


def test_loose_pinv_threshold_is_caught(monkeypatch):
    from scipy import linalg
    p = 5
    x = G.surface_points(p, np.zeros(3), 1.0, G.ALPHA_INNER)
    y = G.surface_points(p, np.zeros(3), 1.0, G.ALPHA_OUTER)
    A = O.laplace(x, y)
    V, _ = O.pinv_factors(A, alpha=1e-6)
    s = np.linalg.svd(A, compute_uv=False)
    assert V.shape[1] != np.sum(s > max(A.shape) * np.finfo(float).eps * s[0])
    assert np.linalg.matrix_rank(linalg.pinv(A)) != V.shape[1]


def _directional_worst_error(directional):
    ops = O.compressed_operators(5, 1e-7)
    d = directional(ops["C"], 1e-5)
    return max(np.linalg.norm(C - Ub @ Vp.T, 2) / np.linalg.norm(C, 2)
               for C, Ub, Vp in zip(ops["C"], d["Ubar"], d["Vbarp"]))


def test_directional_reference_is_within_threshold():
    assert _directional_worst_error(O.directional_operators) < 1e-5


def test_directional_factor_without_sigma_is_caught():
    """Vbar' formed without the singular values (Vbar instead of Vbar Sigmabar)."""
    def bad(C, dir_tol):
        d = O.directional_operators(C, dir_tol)
        d["Vbarp"] = [Vp / np.linalg.norm(Vp, axis=0)[None, :] for Vp in d["Vbarp"]]
        return d
    assert not _directional_worst_error(bad) < 1e-5


def test_directional_swapped_factors_are_caught():
    """Ubar and Vbar' exchanged (C_t^T applied instead of C_t)."""
    def bad(C, dir_tol):
        d = O.directional_operators(C, dir_tol)
        d["Ubar"], d["Vbarp"] = d["Vbarp"], d["Ubar"]
        return d
    assert not _directional_worst_error(bad) < 1e-5



def _check_norm_case(seed=5, p=6, level=3):
    """Locals of a check potential phi from far point sources, and of phi + e with a second far
    field e scaled to 1e-6 of phi: the comparator must report ||e|| / ||phi||, because K_tau
    (K_tau)^+ reproduces a smooth check potential. Built by direct kernel evaluation and the
    pseudo-inverse only; no M2L code."""
    rng = np.random.default_rng(seed)
    w = G.box_width(level)
    x = G.surface_points(p, np.zeros(3), w, G.ALPHA_INNER)
    s1 = rng.random((40, 3)) * w + np.array([3.0 * w, -w, 0.5 * w])
    s2 = rng.random((40, 3)) * w + np.array([-2.5 * w, 2.0 * w, -3.0 * w])
    phi = O.laplace(x, s1) @ rng.random(40)
    e = O.laplace(x, s2) @ rng.standard_normal(40)
    e *= 1e-6 * np.linalg.norm(phi) / np.linalg.norm(e)
    L = M.locals_from_check(p, level, phi[None, None, :])
    Le = M.locals_from_check(p, level, (phi + e)[None, None, :])
    return p, level, L, Le


def test_check_norm_comparator_reports_the_check_potential_difference():
    p, level, L, Le = _check_norm_case()
    assert abs(M.check_norm_error(p, level, L, Le) - 1e-6) < 1e-11
    assert M.check_norm_error(p, level, L, L) == 0.0


def test_check_norm_comparator_with_swapped_radii_is_caught(monkeypatch):
    """The comparator's K_tau built with the two radii exchanged (check points on the outer
    surface, equivalent points on the inner one)."""
    def bad(p, level, root_width=1.0, p_c=None):
        w = G.box_width(level, root_width)
        return O.laplace(G.surface_points(p, np.zeros(3), w, G.ALPHA_OUTER),
                         G.surface_points(p, np.zeros(3), w, G.ALPHA_INNER))
    monkeypatch.setattr(M, "down_check_matrix", bad)
    p, level, L, Le = _check_norm_case()
    assert not abs(M.check_norm_error(p, level, L, Le) - 1e-6) < 1e-11


def test_check_norm_comparator_without_the_kernel_matrix_is_caught(monkeypatch):
    """Locals compared directly (K_tau replaced by the identity): the pseudo-inverse's
    amplification of the small perturbation then shows. (A wrong box width is no mistake here:
    K_tau scales as 1/w, and Eq. 16 is relative.)"""
    monkeypatch.setattr(M, "down_check_matrix", lambda p, level, root_width=1.0, p_c=None: np.eye(G.n_surface(p)))
    p, level, L, Le = _check_norm_case()
    assert not abs(M.check_norm_error(p, level, L, Le) - 1e-6) < 1e-11


def test_per_target_error_finds_one_wrong_box():
    """One wrong box among 4,096 moves the level-wide Eq. 16 by about 1/64 of its own error; the
    per-target maximum reports it whole."""
    rng = np.random.default_rng(2)
    ref = rng.random((4096, 1, 56))
    bad = ref.copy()
    bad[1234, 0] *= 1.5
    assert M.rel_l2_error(ref, bad) < 0.5 / 50
    assert abs(M.max_target_rel_error(ref, bad) - 0.5) < 1e-12
    assert M.max_target_rel_error(ref, ref) == 0.0
