"""Helpers for the GPU parity tests: run the C-ABI path on seeded inputs, and the oracle beside it."""
import numpy as np

from oracle import m2l as M


def levels_of(depth):
    return list(range(2, depth + 1))


def concat(qs, levels):
    return np.concatenate([qs[l].reshape(-1) for l in levels])


def split(flat, sizes, levels, R, n):
    out, off = {}, 0
    for l in levels:
        B = sizes[l]
        out[l] = flat[off:off + B * R * n].reshape(B, R, n)
        off += B * R * n
    return out


def run_gpu(lib, depth, p, qs, keys=None, rank_tol=0.0, form="blas", precision="fp64", output="locals",
            level=-1, R=1, fft_grid=None, accumulate=False, init=None, host=False, dir_tol=None, check_order=None):
    """Apply through the C ABI on cuda:0. qs: {level: (B, R, n) float64}. Returns {level: array}."""
    import torch
    keys = keys or {}
    plan = lib.Plan(depth, p, rank_tol, form=form, precision=precision)
    plan.set(output=output, accumulate=accumulate)
    if fft_grid is not None:
        plan.set(fft_grid=fft_grid)
    if dir_tol is not None:
        plan.set(dir_tol=dir_tol)
    if check_order is not None:
        plan.set(check_order=check_order)
    for l, k in keys.items():
        if k is not None:
            plan.set_boxes(l, np.asarray(k, dtype=np.uint64))
    levels = levels_of(depth) if level == -1 else [level]
    n = plan.n
    n_out = plan.nc if output == "check" else n  # check potentials have n_c values per row
    dt = torch.float64 if precision == "fp64" else torch.float32
    q = torch.from_numpy(concat(qs, levels)).to(dt)
    sizes = {l: qs[l].shape[0] for l in levels}
    rows = sum(sizes.values()) * R
    out0 = (torch.zeros(rows * n_out, dtype=dt) if init is None
            else torch.from_numpy(concat(init, levels)).to(dt))
    if host:
        qd, od = q.contiguous(), out0.clone()
    else:
        qd, od = q.cuda(), out0.cuda()
        plan.set_stream()
    plan.apply(qd, od, level=level, n_rhs=R)
    torch.cuda.synchronize()
    flat = od.cpu().double().numpy()
    res = split(flat, sizes, levels, R, n_out)
    plan.close()
    return res


def oracle_level(p, level, q, keys=None, targets=None):
    """(locals, check potentials at unit box width) for one level from the dense oracle."""
    L, phi = M.m2l_dense(p, level, q, keys=keys, targets=targets)
    return L, phi / (2.0 ** level)
