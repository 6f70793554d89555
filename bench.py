#!/usr/bin/env python
"""M2L interactions/s on GB300 for the 3D Laplace kiFMM (arxiv 2408.07436).

One step = one pass of the whole M2L hot path over the 1M-point workload (uniform cube,
depth 5, p = 6, 1 RHS; levels 2..5, 6,039,504 target/source pairs) in every precision the
library offers for it: BLAS-M2L (SVD truncated at 1e-7) in FP64, FP32 and the split tensor-core
forms TF32x3 and BF16x3, and FFT-M2L in FP64 and FP32. Each variant is one m2l_apply over all
levels (one launch per stage covers every level) through the C ABI.

  value      whole-job M2L interactions/s (pairs x RHS x variants per step / device time per
             step), inputs resident in HBM, L2 flushed between timed steps, CUDA events on the
             launching stream, max over ranks.
  e2e        the same through m2l_apply with pinned HOST buffers (H2D and D2H inside the call).
  roofline   the dominant kernel (longest stage) with its algorithmic work per launch divided
             by its live event-timed launch duration.
  variants   interactions/s, ms and stage times of each variant; the relative error of each
             variant against the FP64 oracle (Eq. 16) is measured in the CPU-baseline leg.
  cpu_baseline  the FP64 oracle (dense definition of Eq. 11 + pseudo-inverse) on a bounded sample
             of target boxes, on this host's cores.

--impl reference times the oracle itself (the CPU program the ratio is taken against).
Multi-GPU (torchrun): every rank runs its own independent instance (weak scaling, no
collective on the data path).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2408_07436_gb300 import workloads as W  # noqa: E402

VARIANTS = ["blas-fp64", "blas-fp32", "blas-tf32x3", "blas-bf16x3", "fft-fp64", "fft-fp32"]
METRIC = "M2L interactions/s and % roofline: mixed+batched vs FP64 GPU at stated rel err"
UNIT = "interactions/s"
WORKLOAD = "laplace3d-m2l uniform-cube 1M points depth5 p6 1rhs blas(rank_tol 1e-7)+fft fp64+fp32+tf32x3+bf16x3"

# Nominal per-GPU figures (GB300) used where no measured peak exists.
NOMINAL_FP64_TFLOPS = 1.25       # FP64 (vector and tensor) dense
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0


def fp32_alu_peak_tflops(mhz=SM_MAX_MHZ):
    return SM_COUNT * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# ---------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------------
def variant_parts(v):
    form, prec = v.split("-")
    return form, prec


def algorithmic_work(plan, form, prec, R):
    """Per-stage algorithmic flops of one application (for the roofline of that stage)."""
    from paper_2408_07436_gb300 import m2l as lib
    n = plan.n
    pairs = plan.pairs(-1)
    rows = plan.rows(-1) * R
    if form == "blas":
        k = plan.query(lib.M2L_Q_RANK)
        r = plan.query(lib.M2L_Q_PINV_RANK)
        return {"compress": 2.0 * n * k * rows, "contract": 2.0 * k * k * pairs * R,
                "expand": 2.0 * (r * k + n * r) * rows}
    F = plan.query(lib.M2L_Q_FREQS)
    g = plan.query(lib.M2L_Q_GRID)
    p = plan.p
    H = g // 2 + 1
    fwd = 8.0 * p * (p * p * H / 2 + p * g * H + g * g * H)
    inv = 8.0 * (p * g * H * g + p * p * H * g) + 4.0 * n * H
    r = plan.query(lib.M2L_Q_PINV_RANK)
    return {"fft_forward": fwd * rows, "hadamard": 8.0 * F * pairs * R, "fft_inverse": inv * rows,
            "pinv": 2.0 * 2 * n * r * rows}


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2408_07436_gb300 import m2l as lib

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wl = W.c2(depth=args.depth)
    R = wl.n_rhs
    variants = args.variants.split(",")
    # every rank draws its own independent instance of the workload
    q64 = np.concatenate([wl.multipoles(l, rng_offset=rank).reshape(-1) for l in wl.levels])
    bufs = {}
    plans = {}
    for v in variants:
        form, prec = variant_parts(v)
        tol = wl.rank_tol if form == "blas" else 0.0
        pl = lib.Plan(wl.depth, wl.p, tol, form=form, precision=prec).set(timing=1)
        pl.set_stream()
        plans[v] = pl
        dt = torch.float64 if prec == "fp64" else torch.float32
        if dt not in bufs:
            bufs[dt] = (torch.from_numpy(q64).to(dt).to(dev), torch.empty(len(q64), dtype=dt, device=dev))
    pairs = plans[variants[0]].pairs(-1)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        for v in variants:
            form, prec = variant_parts(v)
            dt = torch.float64 if prec == "fp64" else torch.float32
            qd, od = bufs[dt]
            plans[v].apply(qd, od, -1, R)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    stage_acc = {v: {} for v in variants}
    var_ms = {v: 0.0 for v in variants}
    launches = 0
    sampler = ClockSampler()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    total_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()  # L2 flush, outside the timed interval
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(variants) + 1)]
        evs[0].record(stream)
        for i, v in enumerate(variants):
            form, prec = variant_parts(v)
            dt = torch.float64 if prec == "fp64" else torch.float32
            qd, od = bufs[dt]
            plans[v].apply(qd, od, -1, R)
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        total_ms += evs[0].elapsed_time(evs[-1])
        for i, v in enumerate(variants):
            var_ms[v] += evs[i].elapsed_time(evs[i + 1])
            for name, (ms, nl) in plans[v].stage_times().items():
                a = stage_acc[v].setdefault(name, [0.0, 0])
                a[0] += ms
                a[1] += nl
                launches += nl
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = sampler.stop()
    ms_step = total_ms / args.steps
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms_step], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    inter_step = pairs * R * len(variants)
    value = world * inter_step / (ms_step / 1e3)

    # roofline of the dominant kernel
    peaks = measured_peaks()
    best = None
    var_out = {}
    for v in variants:
        form, prec = variant_parts(v)
        work = algorithmic_work(plans[v], form, prec, R)
        stages = {}
        for name, (ms, nl) in stage_acc[v].items():
            if nl == 0:
                continue
            per_launch_ms = ms / nl
            flops_launch = work.get(name, 0.0) * args.steps / nl
            stages[name] = {"ms_per_step": ms / args.steps, "launches_per_step": nl / args.steps,
                            "gflops": flops_launch / (per_launch_ms / 1e3) / 1e9 if per_launch_ms > 0 else None}
            if best is None or ms > best[0]:
                best = (ms, v, name, per_launch_ms, flops_launch, prec)
        var_out[v] = {"interactions_per_s": pairs * R / (var_ms[v] / args.steps / 1e3),
                      "ms": var_ms[v] / args.steps, "stages": stages}
        if form == "blas":
            var_out[v]["rank"] = plans[v].query(lib.M2L_Q_RANK)
    def peak_for(prec):
        if prec == "fp64":
            return NOMINAL_FP64_TFLOPS, "alu", "nominal GB300 FP64 1.25 TFLOP/s"
        if prec == "fp32":
            return fp32_alu_peak_tflops(), "alu", "152 SM x 128 FP32 lanes x 2 flops x 2070 MHz"
        bf = peaks.get("bf16_tflops_sustained", 1700.0)
        if prec == "bf16x3":
            return bf / 3.0, "tensor", "of measured: bf16 sustained / 3 (each useful product is 3 MMAs)"
        return bf / 2.0 / 3.0, "tensor", "of measured: bf16 sustained / 2 (nominal tf32 ratio) / 3 (3 MMAs per product)"

    def roof(v, name, ms_total, nl, flops_launch):
        prec = variant_parts(v)[1]
        pk, bound, note = peak_for(prec)
        per_launch_ms = ms_total / nl
        ach = flops_launch / (per_launch_ms / 1e3) / 1e12
        return {"bound": bound, "kernel": f"{v}:{name}", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                "frac": ach / pk, "traffic": None, "peak_source": note}

    for v in variants:
        st = {n: a for n, a in stage_acc[v].items() if a[1] > 0}
        if not st:
            continue
        name = max(st, key=lambda n: st[n][0])
        ms_tot, nl = st[name]
        work = algorithmic_work(plans[v], *variant_parts(v), R)
        var_out[v]["roofline"] = roof(v, name, ms_tot, nl, work.get(name, 0.0) * args.steps / nl)
    _, bv, bname, bms, bflops, bprec = best
    roofline = roof(bv, bname, bms * 1.0, 1, bflops)

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        hq = {dt: torch.from_numpy(q64).to(dt).pin_memory() for dt in bufs}
        ho = {dt: torch.empty(len(q64), dtype=dt).pin_memory() for dt in bufs}
        h2d = d2h = 0
        for v in variants:
            dt = torch.float64 if variant_parts(v)[1] == "fp64" else torch.float32
            plans[v].apply(hq[dt], ho[dt], -1, R)  # warm the staging buffers
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for v in variants:
                dt = torch.float64 if variant_parts(v)[1] == "fp64" else torch.float32
                plans[v].apply(hq[dt], ho[dt], -1, R)
        el = time.perf_counter() - t0
        for v in variants:
            dt = torch.float64 if variant_parts(v)[1] == "fp64" else torch.float32
            h2d += hq[dt].numel() * hq[dt].element_size()
            d2h += ho[dt].numel() * ho[dt].element_size()
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([el], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        e2e = {"value": world * inter_step * args.steps / el, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    mixed = [v for v in variants if variant_parts(v)[1] in ("tf32x3", "bf16x3", "fp32")]
    fp64 = [v for v in variants if variant_parts(v)[1] == "fp64"]
    headline = None
    if mixed and fp64:
        bm = max(mixed, key=lambda v: var_out[v]["interactions_per_s"])
        bf = max(fp64, key=lambda v: var_out[v]["interactions_per_s"])
        headline = {"fastest_reduced_precision": bm, "fastest_fp64": bf,
                    "speedup": var_out[bm]["interactions_per_s"] / var_out[bf]["interactions_per_s"]}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "+".join(sorted({variant_parts(v)[1] for v in variants})), "data": "synthetic",
           "config": {"workload": WORKLOAD, "levels": wl.levels, "pairs_per_variant": pairs, "n_rhs": R,
                      "variants": variants, "l2": "flushed between timed steps (512 MB write)",
                      "instances": "one independent instance per rank"},
           "gpu_launches": launches, "clocks": clocks, "roofline": roofline, "e2e": e2e, "variants": var_out,
           "mixed_vs_fp64": headline}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl, q64, plans, bufs, args.cpu_seconds)
    for pl in plans.values():
        pl.close()
    return out


def _oracle_sample(wl, q64, seconds, seed=11):
    """Run the dense FP64 oracle on random target boxes of every level until `seconds` elapse."""
    from oracle import m2l as M
    n = W.n_surface(wl.p)
    R = wl.n_rhs
    qs, off = {}, 0
    for l in wl.levels:
        B = wl.n_boxes(l)
        qs[l] = q64[off:off + B * R * n].reshape(B, R, n)
        off += B * R * n
    rng = np.random.default_rng(seed)
    done_pairs = 0
    results = {l: ([], [], []) for l in wl.levels}
    t0 = time.perf_counter()
    batches = 0
    while True:
        for l in wl.levels:
            B = wl.n_boxes(l)
            tg = rng.choice(B, size=min(B, 16), replace=False)
            L, phi = M.m2l_dense(wl.p, l, qs[l], targets=tg)
            results[l][0].append(tg)
            results[l][1].append(phi / (2.0 ** l))
            results[l][2].append(L)
            done_pairs += int(M.interaction_csr(l, None, tg)[2][-1])
        batches += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return done_pairs * R, el, results, batches


def cpu_baseline(wl, q64, plans, bufs, seconds):
    """The FP64 oracle on this host's cores, on a bounded sample; also the error of each variant."""
    import torch
    from oracle import m2l as M
    cores = os.cpu_count()
    inter, el, res, batches = _oracle_sample(wl, q64, seconds)
    errs = {}
    n = W.n_surface(wl.p)
    for v, pl in plans.items():
        form, prec = variant_parts(v)
        dt = torch.float64 if prec == "fp64" else torch.float32
        qd, od = bufs[dt]
        pl.set(output="check")
        pl.apply(qd, od, -1, wl.n_rhs)
        chk = od.double().cpu().numpy()
        pl.set(output="locals")
        pl.apply(qd, od, -1, wl.n_rhs)
        loc = od.double().cpu().numpy()
        e_chk, e_loc = [], []
        off = 0
        for l in wl.levels:
            B = wl.n_boxes(l)
            c = chk[off:off + B * wl.n_rhs * n].reshape(B, wl.n_rhs, n)
            lo = loc[off:off + B * wl.n_rhs * n].reshape(B, wl.n_rhs, n)
            tg = np.concatenate(res[l][0])
            ref_phi = np.concatenate(res[l][1])
            ref_L = np.concatenate(res[l][2])
            e_chk.append(M.rel_l2_error(ref_phi, c[tg]))
            e_loc.append(M.check_norm_error(wl.p, l, ref_L, lo[tg]))
            off += B * wl.n_rhs * n
        errs[v] = {"check_potential_rel_err_per_level": e_chk, "locals_rel_err_per_level": e_loc}
    return {"value": inter / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{batches} batches of 16 random target boxes per level of the same workload, dense "
                      f"FP64 definition (per-pair kernel evaluation + pseudo-inverse), {el:.1f} s",
            "rel_err_vs_oracle": errs}


def run_reference(args):
    """The oracle (FP64, this host's cores) timed on bounded samples of the same workload."""
    wl = W.c2()
    q64 = np.concatenate([wl.multipoles(l).reshape(-1) for l in wl.levels])
    per_step = args.ref_seconds
    for _ in range(args.warmup):
        _oracle_sample(wl, q64, per_step / 4)
    tot_inter, tot_el = 0, 0.0
    for i in range(args.steps):
        inter, el, _, _ = _oracle_sample(wl, q64, per_step, seed=100 + i)
        tot_inter += inter
        tot_el += el
    value = tot_inter / tot_el
    cores = os.cpu_count()
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot_el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "levels": wl.levels},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"per step about {per_step:.0f} s of random target boxes (16 per level "
                                       f"per batch) of the same workload, dense FP64 definition"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variants", default=",".join(VARIANTS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-seconds", type=float, default=6.0)
    ap.add_argument("--depth", type=int, default=5, help="tree depth (5 is the workload; smaller for profiling)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    out = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
