"""Octree geometry, kiFMM surfaces and M2L interaction lists (oracle; FP64, plain numpy).

Test infrastructure: see the package docstring for who may import this module.

Readings of the paper used here (the paper is silent or ambiguous on these):
  * Surfaces (Sec. 2.1.1, Fig. 3; App. A.3 surface-point count): the points of a regular
    p x p x p lattice that lie on the boundary of the cube, i.e. 6(p-1)^2 + 2 points.
    Lattice order: (a, b, c) lexicographic with a (the x index) slowest.
    A point is  centre + alpha * (w/2) * (-1 + 2*(a,b,c)/(p-1)).
  * Radii: alpha = 1.05 for the upward-equivalent and downward-check surfaces,
    alpha = 2.95 for the upward-check and downward-equivalent surfaces. The upward
    equivalent and downward check surfaces share one radius, which the convolution view
    of Sec. 2.2 needs.
  * M2L sources (Sec. 2.2): the source box enters through its UPWARD equivalent surface
    (its multipole expansion); the text's "downward equivalent surface of a source box"
    is read as the upward one.
  * Interaction list (Sec. 2, Sec. 2.2): sigma is in I_tau iff parent(sigma) is parent(tau)
    or one of its neighbours, and sigma is not adjacent to tau (max-norm distance of box
    indices >= 2). Non-periodic. Levels 2..depth.
  * Morton key: bit interleave of (x, y, z) box indices with x in the lowest bit of each
    triple. Boxes at a level are stored in ascending Morton order.
"""

from __future__ import annotations

import numpy as np

ALPHA_INNER = 1.05  # upward-equivalent and downward-check surfaces
ALPHA_OUTER = 2.95  # upward-check and downward-equivalent surfaces


def n_surface(p: int) -> int:
    """Number of surface points, written out by counting (compare App. A.3's closed form)."""
    return len(surface_lattice(p))


def surface_lattice(p: int) -> np.ndarray:
    """Integer lattice coordinates (n, 3) of the surface points of order p (Sec. 2.1.1)."""
    if p < 2:
        raise ValueError("expansion order p must be >= 2")
    pts = []
    for a in range(p):
        for b in range(p):
            for c in range(p):
                if a in (0, p - 1) or b in (0, p - 1) or c in (0, p - 1):
                    pts.append((a, b, c))
    return np.array(pts, dtype=np.int64)


def surface_points(p: int, centre, width: float, alpha: float) -> np.ndarray:
    """Physical surface points (n, 3) for a box of side ``width`` centred at ``centre``."""
    lat = surface_lattice(p).astype(np.float64)
    centre = np.asarray(centre, dtype=np.float64)
    return centre[None, :] + alpha * (width / 2.0) * (-1.0 + 2.0 * lat / (p - 1))


def box_width(level: int, root_width: float = 1.0) -> float:
    return root_width / (2 ** level)


def box_centre(idx, level: int, root_origin=(0.0, 0.0, 0.0), root_width: float = 1.0) -> np.ndarray:
    """Centre of the box with integer index ``idx`` (..., 3) at ``level``."""
    w = box_width(level, root_width)
    idx = np.asarray(idx, dtype=np.float64)
    return np.asarray(root_origin, dtype=np.float64) + (idx + 0.5) * w


def morton_encode(idx, level: int) -> np.ndarray:
    """Morton keys of integer box indices (..., 3): bit b of x goes to bit 3b, y to 3b+1, z to 3b+2."""
    idx = np.asarray(idx, dtype=np.int64)
    key = np.zeros(idx.shape[:-1], dtype=np.int64)
    for b in range(level):
        for axis in range(3):
            key |= ((idx[..., axis] >> b) & 1) << (3 * b + axis)
    return key


def morton_decode(key, level: int) -> np.ndarray:
    key = np.asarray(key, dtype=np.int64)
    idx = np.zeros(key.shape + (3,), dtype=np.int64)
    for b in range(level):
        for axis in range(3):
            idx[..., axis] |= ((key >> (3 * b + axis)) & 1) << b
    return idx


def all_boxes(level: int) -> np.ndarray:
    """Integer indices (8^level, 3) of every box at ``level`` in ascending Morton order."""
    return morton_decode(np.arange(8 ** level, dtype=np.int64), level)


def is_adjacent_or_same(a, b) -> bool:
    return int(np.max(np.abs(np.asarray(a) - np.asarray(b)))) <= 1


def interaction_list(tau, level: int, occupied: set | None = None) -> list[tuple[int, int, int]]:
    """I_tau for box index ``tau`` at ``level`` (Sec. 2.2), ascending Morton order.

    Children of the parent's neighbours (the parent itself included) that are not adjacent
    to tau. If ``occupied`` (a set of index tuples) is given, empty sources are dropped
    (the pruning of empty branches, Sec. 2.1).
    """
    n = 2 ** level
    tau = tuple(int(v) for v in tau)
    parent = tuple(v // 2 for v in tau)
    out = []
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                pn = (parent[0] + dx, parent[1] + dy, parent[2] + dz)
                if min(pn) < 0 or max(pn) >= n // 2:
                    continue
                for cx in (0, 1):
                    for cy in (0, 1):
                        for cz in (0, 1):
                            s = (2 * pn[0] + cx, 2 * pn[1] + cy, 2 * pn[2] + cz)
                            if is_adjacent_or_same(s, tau):
                                continue
                            if occupied is not None and s not in occupied:
                                continue
                            out.append(s)
    out.sort(key=lambda s: _morton_scalar(s, level))
    return out


def _morton_scalar(idx, level: int) -> int:
    key = 0
    for b in range(level):
        for axis in range(3):
            key |= ((int(idx[axis]) >> b) & 1) << (3 * b + axis)
    return key


def interaction_lists_vectorised(targets: np.ndarray, level: int, source_slot=None):
    """CSR interaction lists for many targets at once (same rule as ``interaction_list``).

    targets      (T, 3) integer box indices.
    source_slot  optional callable mapping (K, 3) source indices to row numbers (or -1 for
                 an empty box); default is the Morton key (dense level).
    Returns (offsets (T+1,), sources (S, 3), rows (S,)) with, per target, the sources in
    ascending Morton order.
    """
    targets = np.asarray(targets, dtype=np.int64)
    n = 2 ** level
    cand = []
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                for cx in (0, 1):
                    for cy in (0, 1):
                        for cz in (0, 1):
                            cand.append((dx, dy, dz, cx, cy, cz))
    cand = np.array(cand, dtype=np.int64)  # (216, 6)
    parent = targets // 2
    src = 2 * (parent[:, None, :] + cand[None, :, :3]) + cand[None, :, 3:]  # (T, 216, 3)
    pn = parent[:, None, :] + cand[None, :, :3]
    valid = np.all((pn >= 0) & (pn < n // 2), axis=-1)
    valid &= np.max(np.abs(src - targets[:, None, :]), axis=-1) >= 2
    src_c = np.clip(src, 0, n - 1)
    if source_slot is None:
        rows = morton_encode(src_c, level)
    else:
        rows = source_slot(src_c.reshape(-1, 3)).reshape(src_c.shape[:2])
    valid &= rows >= 0
    keys = np.where(valid, morton_encode(src_c, level), np.iinfo(np.int64).max)
    order = np.argsort(keys, axis=1, kind="stable")
    counts = valid.sum(axis=1)
    offsets = np.zeros(len(targets) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(counts)
    sel_src = np.take_along_axis(src_c, order[:, :, None], axis=1)
    sel_rows = np.take_along_axis(rows, order, axis=1)
    sel_valid = np.take_along_axis(valid, order, axis=1)
    return offsets, sel_src[sel_valid], sel_rows[sel_valid]


def transfer_vectors() -> np.ndarray:
    """All transfer vectors t = idx(sigma) - idx(tau) that can occur (Sec. 3.1): [-3,3]^3 minus [-1,1]^3."""
    out = []
    for x in range(-3, 4):
        for y in range(-3, 4):
            for z in range(-3, 4):
                if max(abs(x), abs(y), abs(z)) >= 2:
                    out.append((x, y, z))
    return np.array(out, dtype=np.int64)


def pair_count_closed_form(level: int) -> int:
    """Number of (tau, sigma) M2L pairs on a full non-periodic level, by inclusion-exclusion.

    Pairs whose parents are equal or adjacent (per axis |floor(i/2)-floor(j/2)| <= 1) minus
    pairs that are adjacent or equal (per axis |i-j| <= 1); both conditions factor over the
    three axes, so the count is a^3 - b^3.
    """
    n = 2 ** level
    a = sum(1 for i in range(n) for j in range(n) if abs(i // 2 - j // 2) <= 1)
    b = sum(1 for i in range(n) for j in range(n) if abs(i - j) <= 1)
    return a ** 3 - b ** 3


def occupied_boxes(points: np.ndarray, level: int, root_origin, root_width: float) -> np.ndarray:
    """Sorted Morton keys of the boxes at ``level`` that contain at least one point."""
    idx = np.floor((np.asarray(points) - np.asarray(root_origin)) / box_width(level, root_width)).astype(np.int64)
    idx = np.clip(idx, 0, 2 ** level - 1)
    return np.unique(morton_encode(idx, level))
