"""A tiny complete kiFMM, used only to pin the M2L oracle end to end (oracle; FP64).

Test infrastructure: see the package docstring for who may import this module.

Uniform octree of the given depth with empty branches pruned (Sec. 2.1); upward pass P2M, M2M
and downward pass L2L + M2L, then L2P and P2P at the leaves (Sec. 2, the two-pass procedure).
Every translation forms a check potential and solves for equivalent densities with the
two-factor pseudo-inverse (Sec. 2.1.1, Sec. 2.2, Eqs. 6-11). The result is compared against
direct summation (Eq. 1) with the error of Eq. 16.
"""

from __future__ import annotations

import numpy as np

from . import _cdirect
from . import geometry as G
from . import m2l as M
from . import operators as O


def _leaf_index(points, depth, root_origin, root_width):
    w = G.box_width(depth, root_width)
    idx = np.floor((points - np.asarray(root_origin)) / w).astype(np.int64)
    return np.clip(idx, 0, 2 ** depth - 1)


def direct(points: np.ndarray, charges: np.ndarray) -> np.ndarray:
    """phi_i = sum_{j != i} K(x_i, x_j) q_j (Eq. 1 with sources = targets)."""
    return _cdirect.direct_potential(points, points, charges)


def upward(points, charges, depth, p, root_origin=(0.0, 0.0, 0.0), root_width=1.0, p_c=None):
    """P2M at the leaves and M2M up to level 2. Returns {level: (keys, q (B, 1, n))}.
    ``p_c`` is the order of every check surface (default p)."""
    pc = p if p_c is None else p_c
    leaf = _leaf_index(points, depth, root_origin, root_width)
    lkeys = G.morton_encode(leaf, depth)
    keys = np.unique(lkeys)
    n = G.n_surface(p)
    out = {}
    # P2M: upward check potential from the points, then the upward pseudo-inverse.
    fac = O.up_pinv(p, depth, root_width, p_c=pc)
    w = G.box_width(depth, root_width)
    q = np.zeros((len(keys), 1, n))
    order = np.argsort(lkeys, kind="stable")          # the points of one leaf are one slice
    bounds = np.searchsorted(lkeys[order], keys, side="left")
    ends = np.searchsorted(lkeys[order], keys, side="right")
    for b, key in enumerate(keys):
        sel = order[bounds[b]:ends[b]]
        c = G.box_centre(G.morton_decode(key, depth), depth, root_origin, root_width)
        x = G.surface_points(pc, c, w, G.ALPHA_OUTER)
        phi = O.laplace(x, points[sel]) @ charges[sel]
        q[b, 0] = O.pinv_apply(fac, phi)
    out[depth] = (keys, q)
    # M2M: parent check potential from the children's upward equivalent densities.
    for level in range(depth - 1, 1, -1):
        ckeys, cq = out[level + 1]
        pkeys = np.unique(ckeys >> 3)
        fac = O.up_pinv(p, level, root_width, p_c=pc)
        w = G.box_width(level, root_width)
        wc = G.box_width(level + 1, root_width)
        q = np.zeros((len(pkeys), 1, n))
        for b, key in enumerate(pkeys):
            c = G.box_centre(G.morton_decode(key, level), level, root_origin, root_width)
            x = G.surface_points(pc, c, w, G.ALPHA_OUTER)
            phi = np.zeros(len(x))
            lo, hi = np.searchsorted(ckeys, [key << 3, (key << 3) + 8])   # ckeys is sorted
            for ci in range(lo, hi):
                cc = G.box_centre(G.morton_decode(ckeys[ci], level + 1), level + 1, root_origin, root_width)
                y = G.surface_points(p, cc, wc, G.ALPHA_INNER)
                phi += O.laplace(x, y) @ cq[ci, 0]
            q[b, 0] = O.pinv_apply(fac, phi)
        out[level] = (pkeys, q)
    return out


def fmm(points, charges, depth, p, root_origin=(0.0, 0.0, 0.0), root_width=1.0, m2l=None, p_c=None):
    """Potentials at every point from the full FMM.

    ``m2l(p, level, q, keys)`` may replace the M2L check-potential evaluation (it must return
    check potentials (B, R, n) for all boxes of ``keys``); the default is the dense oracle.
    """
    if depth < 2:
        raise ValueError("depth must be >= 2")
    up = upward(points, charges, depth, p, root_origin, root_width, p_c)
    pc = p if p_c is None else p_c
    n = G.n_surface(p)
    down = {}
    for level in range(2, depth + 1):
        keys, q = up[level]
        if m2l is None:
            phi = M.check_potentials(p, level, q, keys, None, root_origin, root_width, p_c)
        else:
            phi = m2l(p, level, q, keys)
        if level > 2:
            # L2L: the child's downward check potential from the parent's downward equivalent density.
            pkeys, pL = down[level - 1]
            w = G.box_width(level, root_width)
            wp = G.box_width(level - 1, root_width)
            for b, key in enumerate(keys):
                pi = int(np.searchsorted(pkeys, key >> 3))
                c = G.box_centre(G.morton_decode(key, level), level, root_origin, root_width)
                pcen = G.box_centre(G.morton_decode(pkeys[pi], level - 1), level - 1, root_origin, root_width)
                x = G.surface_points(pc, c, w, G.ALPHA_INNER)
                y = G.surface_points(p, pcen, wp, G.ALPHA_OUTER)
                phi[b, 0] += O.laplace(x, y) @ pL[pi, 0]
        down[level] = (keys, M.locals_from_check(p, level, phi, root_width, p_c))
    # L2P and P2P at the leaves.
    keys, L = down[depth]
    leaf = _leaf_index(points, depth, root_origin, root_width)
    lkeys = G.morton_encode(leaf, depth)
    w = G.box_width(depth, root_width)
    out = np.zeros(len(points))
    for b, key in enumerate(keys):
        sel = np.nonzero(lkeys == key)[0]
        idx = G.morton_decode(key, depth)
        c = G.box_centre(idx, depth, root_origin, root_width)
        y = G.surface_points(p, c, w, G.ALPHA_OUTER)
        out[sel] += O.laplace(points[sel], y) @ L[b, 0]
        near = np.all(np.abs(leaf - idx[None, :]) <= 1, axis=1)
        out[sel] += _cdirect.direct_potential(points[sel], points[near], charges[near])
    return out
