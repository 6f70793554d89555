"""GPU parity on physical multipoles: the upward-equivalent densities that the oracle's own P2M and
M2M (Sec. 2.1) give for seeded point clouds, rather than random densities per surface point. These
are the smooth inputs M2L meets inside an FMM. Every form and precision is held to its stated
bound (tests/bounds.py), level-wide (Eq. 16) and per target box."""
import numpy as np
import pytest

from oracle import fmm as F
from oracle import m2l as M
from oracle import operators as O

from bounds import stated
from gpu_util import run_gpu

pytestmark = pytest.mark.gpu

FORMS = [("blas", "fp64"), ("fft", "fp64"), ("blas", "fp32"), ("fft", "fp32"), ("blas", "tf32x3"),
         ("blas", "bf16x3")]


def _upward(points, charges, depth, p, root_origin=(0.0, 0.0, 0.0), root_width=1.0):
    up = F.upward(points, charges, depth, p, root_origin, root_width)
    qs = {l: up[l][1] for l in range(2, depth + 1)}
    keys = {l: (None if len(up[l][0]) == 8 ** l else up[l][0].astype(np.uint64)) for l in range(2, depth + 1)}
    return qs, keys


def _check(lib, p, depth, qs, keys, rank_tol, forms, sample=None, root_width=1.0):
    ops = O.compressed_operators(p, rank_tol, 1.0) if rank_tol > 0 else None
    refs = {}
    for l in range(2, depth + 1):
        B = qs[l].shape[0]
        tg = np.arange(B) if sample is None else np.arange(0, B, max(1, B // sample))
        k = None if keys[l] is None else keys[l].astype(np.int64)
        _, phi = M.m2l_dense(p, l, qs[l], keys=k, targets=tg, root_width=root_width)
        phi_c = None
        if ops is not None:
            _, phi_c = M.m2l_compressed(p, l, qs[l], ops, keys=k, targets=tg)
        refs[l] = (tg, phi * root_width / 2.0 ** l, phi_c)
    for form, prec in forms:
        rt = rank_tol if form == "blas" else 0.0
        chk = run_gpu(lib, depth, p, qs, keys=keys, rank_tol=rt, form=form, precision=prec, output="check")
        bound = 1e-12 if prec == "fp64" else stated(form, prec, p)   # FP64: check potentials
        for l in range(2, depth + 1):
            tg, dense, comp = refs[l]
            ref = comp if (form == "blas" and comp is not None) else dense
            assert M.rel_l2_error(ref, chk[l][tg]) < bound, (form, prec, p, l)
            tb = 1e-11 if prec == "fp64" else 10 * bound
            assert M.max_target_rel_error(ref, chk[l][tg]) < tb, (form, prec, p, l)


def test_physical_multipoles_8000_point_cloud(lib):
    """The 8,000-point cube cloud (depth 3, p = 4) with its charges, full rank, every form."""
    rng = np.random.default_rng(24081)
    pts, q = rng.random((8000, 3)), rng.random(8000)
    qs, keys = _upward(pts, q, 3, 4)
    _check(lib, 4, 3, qs, keys, 0.0, FORMS)


@pytest.mark.parametrize("p", [6, 8])
def test_physical_multipoles_at_higher_order(lib, p):
    """A 40,000-point cube cloud with charges of both signs at depth 3: p = 6 at full rank, p = 8
    at rank 1e-7 (the BLAS forms against the oracle's compressed form at that rank)."""
    rng = np.random.default_rng(24090 + p)
    pts, q = rng.random((40000, 3)), rng.uniform(-1.0, 1.0, 40000)
    qs, keys = _upward(pts, q, 3, p)
    _check(lib, p, 3, qs, keys, 0.0 if p == 6 else 1e-7, FORMS, sample=24)


def test_physical_multipoles_on_a_sphere_surface(lib):
    """Points on a sphere surface in [-1, 1]^3 (most boxes empty, pruned) at depth 4, p = 4."""
    rng = np.random.default_rng(24094)
    v = rng.standard_normal((20000, 3))
    pts = v / np.linalg.norm(v, axis=1, keepdims=True)
    qs, keys = _upward(pts, rng.standard_normal(20000), 4, 4, root_origin=(-1.0, -1.0, -1.0), root_width=2.0)
    assert any(k is not None for k in keys.values())
    _check(lib, 4, 4, qs, keys, 0.0, FORMS, root_width=2.0)
