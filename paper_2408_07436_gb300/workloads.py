"""Seeded synthetic inputs shaped like the paper's workloads (shared by tests, bench and smoke).

This module holds no M2L arithmetic: it draws point clouds and densities from seeded
generators and bins points into octree boxes to decide which boxes are non-empty. Both the
CUDA path and the oracle receive what it returns.

Workloads (seed = 24080 + index):
  c1  8,000 points U[0,1)^3, densities U[0,1), depth 3, p = 4, 1 RHS, full rank.
  c2  1,000,000 points U[0,1)^3, densities U[-1,1], depth 5, p = 6, 1 RHS, rank_tol 1e-7.
  c3  8,000,000 points U[0,1)^3, densities U[0,1), depth 6, p = 8, 1 RHS, BLAS rank_tol 1e-7.
  c4  2,000,000 points on the unit sphere (normalised Gaussian vectors), root [-1,1]^3,
      depth 6, p = 6, 32 RHS, densities N(0,1), empty boxes pruned.
  c5  64 instances: N = round(exp(U[ln 1e4, ln 2e6])) points U[0,1)^3, depth U{3..6},
      p U{4,6,8,10}, 1-8 RHS, densities U[0,1).
The equivalent densities that enter M2L are drawn from the workload's density distribution,
one value per (box, RHS, surface point); M2L is linear, so their values do not change what is
timed and any values exercise every coefficient of the map.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 24080


def n_surface(p: int) -> int:
    """Points on a cube surface discretised by a p^3 lattice, 6(p-1)^2 + 2."""
    return 6 * (p - 1) ** 2 + 2


def _spread_bits(v: np.ndarray, level: int) -> np.ndarray:
    out = np.zeros_like(v)
    for b in range(level):
        out |= ((v >> b) & 1) << (3 * b)
    return out


def morton_keys(idx: np.ndarray, level: int) -> np.ndarray:
    """Morton keys of (..., 3) integer box indices; x occupies the lowest bit of each triple."""
    idx = np.asarray(idx, dtype=np.int64)
    return (_spread_bits(idx[..., 0], level) | (_spread_bits(idx[..., 1], level) << 1)
            | (_spread_bits(idx[..., 2], level) << 2))


@dataclasses.dataclass
class Workload:
    name: str
    depth: int
    p: int
    n_rhs: int
    rank_tol: float
    seed: int
    density: str                       # "u01", "u11" or "normal"
    keys: dict                         # level -> sorted uint64 Morton keys, or None for a full level
    n_points: int = 0
    fft_grid: int | None = None        # convolution grid side of the FFT form (None: 2p)
    dir_tol: float | None = None       # directional recompression threshold of the BLAS form (None: off)

    @property
    def levels(self):
        return list(range(2, self.depth + 1))

    def n_boxes(self, level: int) -> int:
        k = self.keys.get(level)
        return 8 ** level if k is None else len(k)

    def is_sparse(self) -> bool:
        return any(v is not None for v in self.keys.values())

    def multipoles(self, level: int, dtype=np.float64, rng_offset: int = 0) -> np.ndarray:
        """Equivalent densities (B_l, R, n) for one level, seeded per (workload, level)."""
        rng = np.random.default_rng(self.seed * 1000 + level + 97 * rng_offset)
        shape = (self.n_boxes(level), self.n_rhs, n_surface(self.p))
        return _draw(rng, self.density, shape).astype(dtype, copy=False)

    def all_multipoles(self, dtype=np.float64) -> np.ndarray:
        """Levels 2..depth concatenated in ascending order, flattened per level as (B_l, R, n)."""
        return np.concatenate([self.multipoles(l, dtype).reshape(-1) for l in self.levels])


def _draw(rng, density: str, shape):
    if density == "u01":
        return rng.random(shape)
    if density == "u11":
        return rng.uniform(-1.0, 1.0, shape)
    if density == "normal":
        return rng.standard_normal(shape)
    raise ValueError(density)


def occupied_keys(points: np.ndarray, depth: int, origin, width: float) -> dict:
    """Sorted Morton keys of the non-empty boxes at every level 2..depth."""
    n = 2 ** depth
    idx = np.floor((points - np.asarray(origin)) * (n / width)).astype(np.int64)
    idx = np.clip(idx, 0, n - 1)
    leaf = np.unique(morton_keys(idx, depth))
    out = {depth: leaf.astype(np.uint64)}
    cur = leaf
    for level in range(depth - 1, 1, -1):
        cur = np.unique(cur >> 3)
        out[level] = cur.astype(np.uint64)
    return out


def _dense_or_keys(keys: dict, depth: int) -> dict:
    """Replace a level's key list by None when every box of the level is occupied."""
    return {l: (None if len(keys[l]) == 8 ** l else keys[l]) for l in range(2, depth + 1)}


def uniform_cube(name, idx, n_points, depth, p, n_rhs, rank_tol, density, bin_points=True) -> Workload:
    seed = SEED_BASE + idx
    if bin_points:
        rng = np.random.default_rng(seed)
        pts = rng.random((n_points, 3))
        keys = _dense_or_keys(occupied_keys(pts, depth, (0.0, 0.0, 0.0), 1.0), depth)
    else:
        keys = {l: None for l in range(2, depth + 1)}
    return Workload(name, depth, p, n_rhs, rank_tol, seed, density, keys, n_points)


def c1() -> Workload:
    return uniform_cube("c1", 1, 8_000, 3, 4, 1, 0.0, "u01")


def c2(rank_tol: float = 1e-7, depth: int = 5) -> Workload:
    """The 1M-point workload; ``depth`` < 5 gives the same shape on a shallower tree (profiling).

    Its FFT form runs on the (2p-1)^3 grid: the 2p-1 values of the kernel sequence per axis without
    the padding zero, still free of aliasing (App. A.1)."""
    wl = uniform_cube("c2", 2, 1_000_000, depth, 6, 1, rank_tol, "u11")
    wl.fft_grid = 2 * wl.p - 1
    # Eq. 15 at a tenth of the rank threshold: a directional cut adds about ten times its
    # threshold to the compressed check potential, which then stays below the rank truncation's
    wl.dir_tol = rank_tol / 10 if rank_tol > 0 else None
    return wl


def c3(bin_points: bool = True) -> Workload:
    wl = uniform_cube("c3", 3, 8_000_000, 6, 8, 1, 1e-7, "u01", bin_points)
    wl.dir_tol = wl.rank_tol / 10  # as for the 1M-point workload
    return wl


def c4() -> Workload:
    seed = SEED_BASE + 4
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((2_000_000, 3))
    pts = v / np.linalg.norm(v, axis=1, keepdims=True)
    keys = _dense_or_keys(occupied_keys(pts, 6, (-1.0, -1.0, -1.0), 2.0), 6)
    return Workload("c4", 6, 6, 32, 1e-7, seed, "normal", keys, 2_000_000)


def c5_params(n_inst: int = 64):
    """(N, depth, p, n_rhs) of each uneven instance."""
    rng = np.random.default_rng(SEED_BASE + 5)
    out = []
    for _ in range(n_inst):
        n = int(round(math.exp(rng.uniform(math.log(1e4), math.log(2e6)))))
        depth = int(rng.integers(3, 7))
        p = int(rng.choice([4, 6, 8, 10]))
        r = int(rng.integers(1, 9))
        out.append((n, depth, p, r))
    return out


def c5(n_inst: int = 64) -> list:
    out = []
    for i, (n, depth, p, r) in enumerate(c5_params(n_inst)):
        seed = (SEED_BASE + 5) * 100 + i
        rng = np.random.default_rng(seed)
        pts = rng.random((n, 3))
        keys = _dense_or_keys(occupied_keys(pts, depth, (0.0, 0.0, 0.0), 1.0), depth)
        out.append(Workload(f"c5.{i}", depth, p, r, 1e-6, seed, "u01", keys, n))
    return out


def small(depth=3, p=4, n_rhs=1, density="u01", n_points=None, seed=7, rank_tol=0.0) -> Workload:
    """A small workload for tests: full levels unless ``n_points`` points are binned."""
    if n_points is None:
        keys = {l: None for l in range(2, depth + 1)}
    else:
        rng = np.random.default_rng(seed)
        pts = rng.random((n_points, 3))
        keys = _dense_or_keys(occupied_keys(pts, depth, (0.0, 0.0, 0.0), 1.0), depth)
    return Workload(f"small-d{depth}-p{p}-r{n_rhs}", depth, p, n_rhs, rank_tol, seed, density, keys,
                    n_points or 0)
