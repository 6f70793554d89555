"""The M2L translation written out from its definition (oracle; FP64).

Test infrastructure: see the package docstring for who may import this module.

Three independent statements of the same map, each at one level of a uniform octree:
  * ``m2l_dense``       Eq. 11: for each target, sum K_{sigma,tau} q^sigma over I_tau from the
                        actual coordinates (compiled helper ``direct.c``), then the
                        pseudo-inverse of Eqs. 7-10.
  * ``m2l_compressed``  Sec. 3.2 steps 1-5 with the SVD operators of Sec. 3.1 (Eqs. 12-14),
                        then the same pseudo-inverse.
  * ``m2l_fft``         App. A.1: kernel sequences on the 2P convolution grid, FFT of the
                        embedded densities, Hadamard products summed over I_tau, inverse FFT.
                        The paper's steps 3 and 5 (interleave into / out of frequency order)
                        only rearrange memory and are not written out.

Box sets: ``keys=None`` means the full level (8^l boxes in ascending Morton order);
otherwise ``keys`` is the sorted array of Morton keys of the non-empty boxes and the
multipole rows follow that order. Empty boxes are neither targets nor sources (Sec. 2.1).
Densities are arrays (B, R, n): box, right-hand side, surface point.
"""

from __future__ import annotations

import numpy as np

from . import _cdirect
from . import geometry as G
from . import operators as O


def _boxes_and_slot(level: int, keys):
    if keys is None:
        boxes = G.all_boxes(level)

        def slot(idx):
            return G.morton_encode(idx, level)
    else:
        keys = np.asarray(keys, dtype=np.int64)
        boxes = G.morton_decode(keys, level)

        def slot(idx):
            k = G.morton_encode(idx, level)
            pos = np.searchsorted(keys, k)
            pos_c = np.clip(pos, 0, len(keys) - 1)
            return np.where((pos < len(keys)) & (keys[pos_c] == k), pos_c, -1)
    return boxes, slot


def interaction_csr(level: int, keys=None, targets=None):
    """(target rows, offsets, source index triples, source rows) for the requested targets."""
    boxes, slot = _boxes_and_slot(level, keys)
    rows = np.arange(len(boxes)) if targets is None else np.asarray(targets, dtype=np.int64)
    offsets, src, srow = G.interaction_lists_vectorised(boxes[rows], level, slot)
    return rows, boxes, offsets, src, srow


def m2l_surfaces(p: int, width: float, p_c: int | None = None):
    """Offsets from the box centre of the target's downward-check points (order p_c, default p)
    and the source's upward-equivalent points (Sec. 2.2); both lie on the inner radius."""
    x_off = G.surface_points(p if p_c is None else p_c, np.zeros(3), width, G.ALPHA_INNER)
    y_off = G.surface_points(p, np.zeros(3), width, G.ALPHA_INNER)
    return x_off, y_off


def check_potentials(p: int, level: int, q: np.ndarray, keys=None, targets=None,
                     root_origin=(0.0, 0.0, 0.0), root_width: float = 1.0, p_c: int | None = None) -> np.ndarray:
    """phi_tau = sum_{sigma in I_tau} K_{sigma,tau} q^sigma (the sum in Eq. 11), shape (T, R, n_c)."""
    rows, boxes, offsets, src, srow = interaction_csr(level, keys, targets)
    w = G.box_width(level, root_width)
    x_off, y_off = m2l_surfaces(p, w, p_c)
    t_centre = G.box_centre(boxes[rows], level, root_origin, root_width)
    s_centre = G.box_centre(src, level, root_origin, root_width)
    return _cdirect.check_potential(x_off, y_off, t_centre, offsets, s_centre, srow, q, q.shape[1])


def locals_from_check(p: int, level: int, phi: np.ndarray, root_width: float = 1.0,
                      p_c: int | None = None) -> np.ndarray:
    """q^tau = (K_tau)^+ phi_tau with the two-factor pseudo-inverse (Eqs. 7-10); phi (T, R, n_c)."""
    fac = O.down_pinv(p, level, root_width, p_c=p_c)
    T, R, nc = phi.shape
    cols = phi.reshape(T * R, nc).T
    return O.pinv_apply(fac, cols).T.reshape(T, R, -1)


def m2l_dense(p: int, level: int, q: np.ndarray, keys=None, targets=None,
              root_origin=(0.0, 0.0, 0.0), root_width: float = 1.0, p_c: int | None = None):
    """Eq. 11 at one level. Returns (locals (T,R,n), check potentials (T,R,n_c))."""
    phi = check_potentials(p, level, q, keys, targets, root_origin, root_width, p_c)
    return locals_from_check(p, level, phi, root_width, p_c), phi


def m2l_compressed(p: int, level: int, q: np.ndarray, ops: dict, keys=None, targets=None,
                   root_width: float = 1.0, p_c: int | None = None):
    """BLAS-M2L of Sec. 3.2.

    ``ops`` comes from ``operators.compressed_operators(p, rank_tol, width)`` built at this
    level's box width. When it also holds the directional factors of Eq. 15 (the entries of
    ``operators.directional_operators`` merged in), step 4 applies them as the two products
    xi = Vbar'_t^T q~ and phi~ += Ubar_t xi. Returns (locals, check potentials), shapes (T, R, n).
    """
    rows, boxes, offsets, src, srow = interaction_csr(level, keys, targets)
    U, S, C, tv = ops["U"], ops["S"], ops["C"], ops["tvecs"]
    B, R, n = q.shape
    kc = ops.get("kc", ops["k"])
    # Step 1: map every (target, source) pair to its transfer vector t = idx(sigma) - idx(tau).
    tgt_of_pair = np.repeat(np.arange(len(rows)), np.diff(offsets))
    tvec = src - boxes[rows][tgt_of_pair]
    tindex = {tuple(v): i for i, v in enumerate(tv)}
    t_of_pair = np.array([tindex[tuple(v)] for v in tvec], dtype=np.int64)
    # Step 2: compressed multipoles of every source box, q~ = S^T q.
    qt = q @ S
    # Steps 3-5: per transfer vector, gather its sources, apply C_t, accumulate into targets.
    phit = np.zeros((len(rows), R, kc))
    for ti in range(len(tv)):
        sel = np.nonzero(t_of_pair == ti)[0]
        if len(sel) == 0:
            continue
        gathered = qt[srow[sel]]                       # (N_t, R, k)
        if "Ubar" in ops:
            xi = gathered @ ops["Vbarp"][ti]              # (N_t, R, k_t)
            contrib = xi @ ops["Ubar"][ti].T
        else:
            contrib = gathered @ C[ti].T
        np.add.at(phit, tgt_of_pair[sel], contrib)
    # Uncompress the check potentials, phi = U phi~, then recover the locals.
    phi = phit @ U.T
    return locals_from_check(p, level, phi, root_width, p_c), phi


def kernel_spectra(p: int, width: float, g: int | None = None) -> dict:
    """App. A.1 step 1: real FFT of the kernel grid of every transfer vector."""
    return {tuple(t): np.fft.rfftn(O.kernel_grid(p, t, width, g)) for t in G.transfer_vectors()}


def m2l_fft(p: int, level: int, q: np.ndarray, keys=None, targets=None, root_width: float = 1.0,
            g: int | None = None):
    """FFT-M2L of App. A.1 at one level. Returns (locals, check potentials)."""
    g = O.conv_grid_size(p) if g is None else g
    rows, boxes, offsets, src, srow = interaction_csr(level, keys, targets)
    w = G.box_width(level, root_width)
    spectra = kernel_spectra(p, w, g)
    B, R, n = q.shape
    # Step 2: embed every source density on the convolution grid and transform it.
    needed = np.unique(srow)
    qhat = {int(s): [np.fft.rfftn(O.embed_density(p, q[s, r], g)) for r in range(R)] for s in needed}
    phi = np.zeros((len(rows), R, n))
    for ti in range(len(rows)):
        tau = boxes[rows[ti]]
        for r in range(R):
            acc = np.zeros_like(next(iter(spectra.values())))
            # Step 4: Hadamard products with the kernel spectra, summed over I_tau.
            for e in range(offsets[ti], offsets[ti + 1]):
                t = tuple(int(v) for v in (src[e] - tau))
                acc = acc + spectra[t] * qhat[int(srow[e])][r]
            # Step 6: inverse transform, read the check surface.
            phi[ti, r] = O.extract_surface(p, np.fft.irfftn(acc, s=(g, g, g), axes=(0, 1, 2)))
    return locals_from_check(p, level, phi, root_width), phi


def rel_l2_error(ref: np.ndarray, approx: np.ndarray) -> float:
    """Relative L2 error of Eq. 16."""
    ref = np.asarray(ref, dtype=np.float64)
    approx = np.asarray(approx, dtype=np.float64)
    den = np.sum(np.abs(ref) ** 2)
    num = np.sum(np.abs(ref - approx) ** 2)
    return float(np.sqrt(num / den)) if den > 0 else float(np.sqrt(num))


def max_target_rel_error(ref: np.ndarray, approx: np.ndarray) -> float:
    """Largest relative L2 error of one target's values: max over (box, rhs) of
    ||ref[b, r] - approx[b, r]|| / ||ref[b, r]|| (Eq. 16 per target box and right-hand side).
    A single wrong box among many barely moves the level-wide error of Eq. 16; here it is the
    maximum."""
    ref = np.asarray(ref, dtype=np.float64)
    approx = np.asarray(approx, dtype=np.float64)
    num = np.sqrt(np.sum((ref - approx) ** 2, axis=-1))
    den = np.sqrt(np.sum(ref ** 2, axis=-1))
    rel = np.where(den > 0, num / np.where(den > 0, den, 1.0), num)
    return float(rel.max()) if rel.size else 0.0


def down_check_matrix(p: int, level: int, root_width: float = 1.0, p_c: int | None = None) -> np.ndarray:
    """K_tau: the downward-equivalent surface of a box of ``level`` seen from its own downward
    check surface (the matrix of Eq. 6 that the locals solve with, Sec. 2.2)."""
    w = G.box_width(level, root_width)
    x = G.surface_points(p if p_c is None else p_c, np.zeros(3), w, G.ALPHA_INNER)
    y = G.surface_points(p, np.zeros(3), w, G.ALPHA_OUTER)
    return O.laplace(x, y)


def check_norm_error(p: int, level: int, L_ref: np.ndarray, L_test: np.ndarray, root_width: float = 1.0,
                     p_c: int | None = None) -> float:
    """Eq. 16 applied to the check potentials K_tau q^tau that two sets of locals reproduce.

    The locals solve an ill-conditioned least-squares problem (Sec. 2.1.1), so rounding in the
    check potential is amplified in the locals by up to the condition number of K_tau, and damped
    again whenever the locals are used to evaluate a potential (the footnote of Sec. 2.1.1).
    Comparing K_tau q^tau measures agreement in the quantity the FMM uses downstream.
    """
    K = down_check_matrix(p, level, root_width, p_c)
    a = np.einsum("ij,brj->bri", K, np.asarray(L_ref, dtype=np.float64))
    b = np.einsum("ij,brj->bri", K, np.asarray(L_test, dtype=np.float64))
    return rel_l2_error(a, b)


def locals_backward_bound(p: int, level: int, L: np.ndarray, root_width: float = 1.0,
                          p_c: int | None = None) -> float:
    """How far two correct sets of FP64 locals may sit apart in the check norm of
    ``check_norm_error``: b = n_c eps ||K_tau||_2 ||L|| / ||K_tau L|| (norms over every box and
    right-hand side of ``L``).

    The locals solve K_tau q = phi through the two factors of the pseudo-inverse (Eqs. 7-10 and
    the footnote of Sec. 2.1.1). A normwise backward-stable solve returns the exact solution of a
    matrix within n_c eps ||K_tau|| of K_tau, so its check potential K_tau q differs from another
    such solve's by up to about n_c eps ||K_tau|| ||q||: small against ||phi|| when the locals
    are smooth, large when they oscillate (p >= 8, where cond(K_tau) reaches 1e12)."""
    K = down_check_matrix(p, level, root_width, p_c)
    L = np.asarray(L, dtype=np.float64)
    KL = np.einsum("ij,brj->bri", K, L)
    den = np.linalg.norm(KL)
    if den == 0:
        return 0.0
    return float(K.shape[0] * np.finfo(np.float64).eps * np.linalg.norm(K, 2) * np.linalg.norm(L) / den)


def pair_count(level: int, keys=None) -> int:
    """Number of M2L (target, source) pairs at a level: the sum of |I_tau| over targets."""
    _, _, offsets, _, _ = interaction_csr(level, keys)
    return int(offsets[-1])
