#!/usr/bin/env python
"""M2L interactions/s on GB300 for the 3D Laplace kiFMM (arxiv 2408.07436).

Default workload: 8M points uniform in the unit cube, depth 6 (262,144 leaves), p = 8 (296 surface
points), 1 RHS: M2L at levels 2..6, 52,337,880 target/source pairs per pass.

One step = one m2l_apply over all levels (every stage of the chosen form) through the C ABI, in
the form and precision the library's autotuner picks among the reduced-precision forms whose
stated relative error bound (p-dependent, Eq. 16 on the check potential) and rank truncation
are within the target (default 1e-6). Nothing else runs in the timed region.

  value          interactions/s of that one form: pairs x RHS / device time per step (CUDA events
                 on the launching stream), inputs resident in HBM, L2 flushed between steps.
  fp64_same_target  the FP64 form the autotuner picks at the same target, timed the same way;
                 mixed_vs_fp64 = value / its rate.
  variants       every explicit (form, precision) of the workload, timed alone (not in `value`).
  batched        (default workload) the 64 uneven instances in one graph-replayed, autotuned
                 m2l_apply_batch at the same target.
  e2e            the headline form through m2l_apply with pinned HOST buffers (H2D and D2H
                 inside the call).
  roofline       the dominant kernel of the headline form: algorithmic work per launch divided
                 by its event-timed launch duration, against the measured peak of its pipe
                 (CUDA-core peaks from the FMA probe run at the start of this bench).
  cpu_baseline   the FP64 oracle (dense Eq. 11 + pseudo-inverse) on a bounded sample of target
                 boxes on this host's cores; the same leg measures the relative error of every
                 timed form against it (per level, check potentials and locals).

--impl reference times the oracle itself: the reference arm, a deliberately simple FP64 CPU program.
Multi-GPU (torchrun): every rank runs its own independent instance (weak scaling, no collective on
the data path).
"""

from __future__ import annotations

import argparse
import hashlib
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

METRIC = "M2L interactions/s and % roofline: mixed+batched vs FP64 GPU at stated rel err"
UNIT = "interactions/s"
DEFAULT_TARGET = 1e-6

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a dominant kernel from
# one ncu capture, keyed by (workload, depth, kernel), with the SHA-256 of the source file the
# kernel was built from; the summary and the command are in profiles/. A source that has changed
# since the capture reports null.
TRAFFIC = {
    # hadamard_tc_kernel<4> at level 5 (4,096 clusters, F = 2304): 696,227,072 B read + 556,734,720 B
    # written in one launch; scaled by the clusters of levels 2-6 (9.1426 x level 5's) over the
    # stage's 5 launches (the ncu summary is under profiles/)
    ("c3", 6, "fft-tf32x3:hadamard"): {
        "bytes": 2291060214, "source": "paper_2408_07436_gb300/csrc/hadamard_tc.cu",
        "sha256": "634595ece5aac69450f819203183e8228ce1093701558acbf8a82052877856ef"},
}


def measured_traffic(workload, depth, kernel):
    t = TRAFFIC.get((workload, depth, kernel))
    if not t or t["bytes"] is None:
        return None
    try:
        with open(os.path.join(ROOT, t["source"]), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != t["sha256"]:
                return None
    except OSError:
        return None
    return t["bytes"]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def alu_peaks():
    """FP64 and FP32 FMA throughput of this GPU (TFLOP/s), measured now by the FMA probe."""
    from paper_2408_07436_gb300 import peaks
    out = {}
    for name, fp64, iters in (("fp64", True, 24_000), ("fp32", False, 1_200_000)):
        best, med, ms = peaks.m2l_fma_peak(fp64, iters, reps=5)
        out[name] = {"best_tflops": best, "median_tflops": med, "launch_ms": ms}
    return out


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


def log(msg):
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


# ---------------------------------------------------------------------------------------------
def form_name(lib, f):
    return {lib.M2L_FORM_BLAS: "blas", lib.M2L_FORM_FFT: "fft"}[f]


def prec_name(lib, pr):
    return {lib.M2L_PREC_FP64: "fp64", lib.M2L_PREC_FP32: "fp32", lib.M2L_PREC_TF32X3: "tf32x3",
            lib.M2L_PREC_BF16X3: "bf16x3"}[pr]


def resolved(lib, pl, R):
    """(form, precision) names the plan's next apply with R right-hand sides runs."""
    return form_name(lib, pl.query(lib.M2L_Q_FORM, R)), prec_name(lib, pl.query(lib.M2L_Q_PRECISION, R))


def algorithmic_work(plan, form, R):
    """Per-stage algorithmic flops of one application (for the roofline of that stage). `plan` has
    an explicit form and precision."""
    from paper_2408_07436_gb300 import m2l as lib
    n = plan.n
    pairs = plan.pairs(-1)
    rows = plan.rows(-1) * R
    if form == "blas":
        k = plan.query(lib.M2L_Q_RANK)
        r = plan.query(lib.M2L_Q_PINV_RANK)
        return {"compress": 2.0 * n * k * rows, "contract": float(plan.query(lib.M2L_Q_CONTRACT_FLOPS, -1)) * R,
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


DESC = {
    "c2": "laplace3d-m2l uniform-cube 1M points depth5 p6 1rhs (blas rank_tol 1e-7; fft grid 11^3)",
    "c3": "laplace3d-m2l uniform-cube 8M points depth6 p8 1rhs (blas rank_tol 1e-7; fft grid 16^3)",
    "c4": "laplace3d-m2l unit-sphere-surface 2M points depth6 p6 32rhs, empty boxes pruned (blas rank_tol 1e-7)",
    "c5": "laplace3d-m2l 64 uneven instances (1e4..2e6 points, depth 3-6, p 4/6/8/10, 1-8 rhs), one batched "
          "graph-replayed pass",
}


def workload_spec(name, depth):
    """(instances, explicit variants timed beside the headline, batched) of a named workload."""
    if name == "c2":
        return [W.c2(depth=depth)], ["blas-fp64", "blas-fp32", "blas-tf32x3", "blas-bf16x3", "fft-fp64",
                                     "fft-tf32x3", "fft-fp32"], False
    if name == "c3":
        return [W.c3()], ["blas-bf16x3", "blas-tf32x3", "blas-fp32", "blas-fp64", "fft-tf32x3", "fft-fp32",
                          "fft-fp64"], False
    if name == "c4":
        return [W.c4()], ["blas-bf16x3", "blas-tf32x3", "fft-fp32"], False
    if name == "c5":
        return W.c5(), [], True
    raise ValueError(name)


def make_plan(lib, wl, form, prec, target=None, timing=True, rank_tol=None):
    """A plan of one instance with the workload's options, on the current torch stream. With a
    target the library also picks the BLAS form's rank threshold (M2L_OPT_RANK_AUTO); `rank_tol`
    overrides the workload's threshold."""
    tol = (wl.rank_tol if rank_tol is None else rank_tol) if form in ("blas", "auto") else 0.0
    pl = lib.Plan(wl.depth, wl.p, tol, form=form, precision=prec).set(timing=int(timing))
    if target is not None and form in ("blas", "auto"):
        pl.set(rank_auto=1)
    if form in ("fft", "auto") and wl.fft_grid:
        pl.set(fft_grid=wl.fft_grid)
    if form in ("blas", "auto") and prec in ("fp64", "fp32", "auto") and wl.dir_tol:
        pl.set(dir_tol=wl.dir_tol)  # the CUDA-core contraction applies Eq. 15's factors
    if target is not None:
        pl.set(target_tol=target)
    for l in wl.levels:
        if wl.keys[l] is not None:
            pl.set_boxes(l, wl.keys[l])
    pl.set_stream()
    return pl


class Timed:
    """Device time per step of `run` (CUDA events on the current stream, L2 flushed before each
    step outside the timed interval), with the stage times and launches of the plans it reports."""

    def __init__(self, torch, flush):
        self.torch, self.flush = torch, flush

    def __call__(self, run, steps, warmup, plans=(), sampler=None, barrier=None):
        torch = self.torch
        for _ in range(warmup):
            run()
        torch.cuda.synchronize()
        if barrier:
            barrier()
        if sampler:
            sampler.start()
        stream = torch.cuda.current_stream()
        ms, stages, launches = [], {}, 0
        for _ in range(steps):
            self.flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            run()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
            for pl in plans:
                st = pl.stage_times()
                for name, (sms, nl) in st.items():
                    acc = stages.setdefault(name, [0.0, 0])
                    acc[0] += sms
                    acc[1] += nl
                launches += pl.query(pl_launches_key())
        clocks = sampler.stop() if sampler else None
        if barrier:
            barrier()
        return ms, stages, launches, clocks


def pl_launches_key():
    from paper_2408_07436_gb300 import m2l as lib
    return lib.M2L_Q_LAUNCHES


def roofline_of(lib, wl, form, prec, stages, steps, peaks, alu, args, rank_tol=None):
    """Roofline of the dominant stage (longest device time) of one explicit (form, precision)."""
    if not stages:
        return None
    acct = make_plan(lib, wl, form, prec, timing=False, rank_tol=rank_tol)   # host-side queries (operators shared)
    if rank_tol is not None and wl.dir_tol and prec in ("fp64", "fp32") and form == "blas":
        acct.set(dir_tol=rank_tol / 10)   # the directional threshold follows the chosen rank
    work = algorithmic_work(acct, form, wl.n_rhs)
    acct.close()
    name = max(stages, key=lambda n: stages[n][0])
    ms_tot, nl = stages[name]
    per_launch_ms = ms_tot / nl
    ach = work.get(name, 0.0) * steps / nl / (per_launch_ms / 1e3) / 1e12
    bf = peaks.get("bf16_tflops_sustained")
    if prec in ("fp64", "fp32"):
        pk = alu[prec]["best_tflops"]
        bound, src = "alu", f"measured: {prec.upper()} FMA probe of this run (best of 5 launches of " \
                            f"{alu[prec]['launch_ms']:.0f} ms)"
    elif bf is None:
        pk, bound, src = (1700.0 / 3 if prec == "bf16x3" else 1700.0 / 6), "tensor", \
            "of fallback: 1.7 PFLOP/s bf16 sustained / 3 MMAs per useful product" + (" / 2 (tf32)" if prec == "tf32x3" else "")
    elif form == "fft" and prec == "tf32x3":
        pk, bound, src = bf / 6.0, "tensor", "of measured: bf16 sustained / 6 (the Hadamard's six BF16 piece products per useful one)"
    elif prec == "bf16x3":
        pk, bound, src = bf / 3.0, "tensor", "of measured: bf16 sustained / 3 (each useful product is 3 MMAs)"
    else:
        pk, bound, src = bf / 6.0, "tensor", "of measured: bf16 sustained / 2 (nominal tf32 ratio) / 3 (3 MMAs per product)"
    return {"bound": bound, "kernel": f"{form}-{prec}:{name}", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
            "frac": ach / pk, "traffic": measured_traffic(args.workload, wl.depth, f"{form}-{prec}:{name}"),
            "peak_source": src, "algorithmic_flops_per_launch": work.get(name, 0.0) * steps / nl,
            "launch_ms": per_launch_ms}


def stage_summary(stages, steps):
    return {name: {"ms_per_step": ms / steps, "launches_per_step": nl / steps} for name, (ms, nl) in stages.items()
            if nl}


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2408_07436_gb300 import m2l as lib

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    target = args.target
    insts, variants, batched = workload_spec(args.workload, args.depth)
    if args.variants is not None:
        variants = [v for v in args.variants.split(",") if v]
    alu = alu_peaks()
    log(f"FMA probe: fp64 {alu['fp64']['best_tflops']:.3f} TFLOP/s, fp32 {alu['fp32']['best_tflops']:.1f} TFLOP/s")
    peaks = measured_peaks()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    timed = Timed(torch, flush)
    barrier = None
    if world > 1:
        import torch.distributed as dist
        barrier = dist.barrier
    # every rank draws its own independent instances of the workload
    q64 = [np.concatenate([wl.multipoles(l, rng_offset=rank).reshape(-1) for l in wl.levels]) for wl in insts]
    dbufs = {}

    def buf(i, dt):
        if (i, dt) not in dbufs:
            dbufs[(i, dt)] = (torch.from_numpy(q64[i]).to(dt).to(dev), torch.empty(len(q64[i]), dtype=dt, device=dev))
        return dbufs[(i, dt)]

    def dtype_of(pl, wl):
        return torch.float64 if pl.query(lib.M2L_Q_PRECISION, wl.n_rhs) == lib.M2L_PREC_FP64 else torch.float32

    def runner(plans):
        """One pass over every instance with `plans` (a batch when the workload is batched)."""
        if batched:
            qs = [buf(i, dtype_of(pl, wl))[0] for i, (pl, wl) in enumerate(zip(plans, insts))]
            os_ = [buf(i, dtype_of(pl, wl))[1] for i, (pl, wl) in enumerate(zip(plans, insts))]
            hs, qp, op, rs = ([pl.handle for pl in plans], [q.data_ptr() for q in qs], [o.data_ptr() for o in os_],
                              [wl.n_rhs for wl in insts])

            def run():
                rc = lib.m2l_apply_batch(hs, qp, op, rs)
                if rc != lib.M2L_OK:
                    raise lib.M2LError(rc, lib.m2l_last_error())
            return run
        bs = [buf(i, dtype_of(pl, wl)) for i, (pl, wl) in enumerate(zip(plans, insts))]

        def run():
            for (qd, od), pl, wl in zip(bs, plans, insts):
                pl.apply(qd, od, -1, wl.n_rhs)
        return run

    pairs = [make_plan(lib, wl, "fft", "fp64", timing=False) for wl in insts]
    inter = sum(p_.pairs(-1) * wl.n_rhs for p_, wl in zip(pairs, insts))
    for p_ in pairs:
        p_.close()

    # ---- headline: the autotuned reduced-precision form at the target ----
    if args.headline:
        # fixed form (for profiling: under a profiler the tuner's timings, so its choice, change)
        hf, hp = args.headline.split("-")
        head = [make_plan(lib, wl, hf, hp, timing=not batched) for wl in insts]
    else:
        head = [make_plan(lib, wl, "auto", "auto", target=target, timing=not batched) for wl in insts]
    forms = [resolved(lib, pl, wl.n_rhs) for pl, wl in zip(head, insts)]
    log(f"headline forms at {target:g}: {sorted(set(forms))}")
    run_head = runner(head)
    ms, stages, launches, clocks = timed(run_head, args.steps, args.warmup, plans=[] if batched else head,
                                         sampler=ClockSampler(), barrier=barrier)
    ms_step = sum(ms) / len(ms)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms_step], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    if batched:
        launches = head[0].query(lib.M2L_Q_LAUNCHES) * args.steps
    value = world * inter / (ms_step / 1e3)
    log(f"headline: {ms_step:.2f} ms per step, {value:.3e} interactions/s")
    head_form, head_prec = forms[0] if len(set(forms)) == 1 else ("mixed", "mixed")
    head_rank = None
    if not batched and head_form == "blas":
        head_rank = {"rank_tol": head[0].current_rank_tol(), "k": head[0].query(lib.M2L_Q_RANK)}
    roofline = None
    if not batched:
        roofline = roofline_of(lib, insts[0], head_form, head_prec, stages, args.steps, peaks, alu, args,
                               rank_tol=head_rank["rank_tol"] if head_rank else None)

    # ---- the FP64 form the autotuner picks at the same target ----
    fp64_out, fp64_plans = None, None
    if not args.no_fp64:
        fp64_plans = [make_plan(lib, wl, "auto", "fp64", target=target, timing=not batched) for wl in insts]
        f64 = [resolved(lib, pl, wl.n_rhs) for pl, wl in zip(fp64_plans, insts)]
        k = max(1, min(args.steps, 3))
        ms64, st64, _, _ = timed(runner(fp64_plans), k, 2, plans=[] if batched else fp64_plans, barrier=barrier)
        m64 = sum(ms64) / len(ms64)
        fp64_out = {"interactions_per_s": world * inter / (m64 / 1e3), "ms": m64, "steps": k,
                    "forms": sorted(set(f"{a}-{b}" for a, b in f64)), "stages": stage_summary(st64, k)}
        if not batched and f64[0][0] == "blas":
            fp64_out["rank"] = {"rank_tol": fp64_plans[0].current_rank_tol(), "k": fp64_plans[0].query(lib.M2L_Q_RANK)}
        if not batched:
            fp64_out["roofline"] = roofline_of(lib, insts[0], f64[0][0], f64[0][1], st64, k, peaks, alu, args,
                                               rank_tol=fp64_out.get("rank", {}).get("rank_tol"))
        log(f"fp64 at {target:g}: {fp64_out['forms']} {m64:.1f} ms")

    # ---- every explicit variant of the workload, alone ----
    var_out, var_plans = {}, {}
    for v in variants:
        form, prec = v.split("-")
        pls = [make_plan(lib, wl, form, prec, timing=True) for wl in insts]
        try:
            mv, sv, _, _ = timed(runner(pls), 2, 1, plans=pls)
        except lib.M2LError as e:
            var_out[v] = {"unavailable": str(e)}
            for pl in pls:
                pl.close()
            continue
        m = sum(mv) / len(mv)
        var_out[v] = {"interactions_per_s": world * inter / (m / 1e3), "ms": m, "steps": 2,
                      "stages": stage_summary(sv, 2),
                      "roofline": roofline_of(lib, insts[0], form, prec, sv, 2, peaks, alu, args)}
        if form == "blas":
            var_out[v]["rank"] = pls[0].query(lib.M2L_Q_RANK)
        var_plans[v] = pls
        log(f"variant {v}: {m:.2f} ms")

    # ---- the 64 uneven instances in one batched pass (extra key of the default workload) ----
    batch_out = None
    if args.workload == "c3" and not args.no_batch:
        batch_out = run_batched_key(lib, torch, timed, dev, target, rank)
        log(f"batched: {batch_out['ms']:.1f} ms per pass")

    # ---- end to end through the C ABI with pinned host buffers ----
    e2e = None
    if not args.no_e2e:
        hq, ho = {}, {}
        for i, (pl, wl) in enumerate(zip(head, insts)):
            dt = dtype_of(pl, wl)
            hq[i] = torch.from_numpy(q64[i]).to(dt).pin_memory()
            ho[i] = torch.empty_like(hq[i]).pin_memory()

        def e2e_pass():
            if batched:
                for i, (pl, wl) in enumerate(zip(head, insts)):
                    buf(i, dtype_of(pl, wl))[0].copy_(hq[i], non_blocking=True)
                run_head()
                for i, (pl, wl) in enumerate(zip(head, insts)):
                    ho[i].copy_(buf(i, dtype_of(pl, wl))[1], non_blocking=True)
                torch.cuda.synchronize()
            else:
                for i, (pl, wl) in enumerate(zip(head, insts)):
                    pl.apply(hq[i], ho[i], -1, wl.n_rhs)   # host pointers: staged inside the call

        e2e_pass()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_pass()
        el = time.perf_counter() - t0
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([el], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        nbytes = sum(hq[i].numel() * hq[i].element_size() for i in hq)
        e2e = {"value": world * inter * args.steps / el, "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes}
        log("e2e done")

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": head_prec, "data": "synthetic",
           "config": {"workload": DESC[args.workload] if args.depth == 5 or args.workload != "c2"
                      else DESC["c2"].replace("depth5", f"depth{args.depth}"),
                      "instances": len(insts), "pairs_x_rhs": int(inter), "target_rel_err": target,
                      "form": head_form, "precision": head_prec, "rank": head_rank,
                      "choice": (f"fixed by --headline {args.headline}" if args.headline else
                                 "autotuned among forms whose stated bound plus estimated rank truncation is within "
                                 "the target, BLAS rank threshold chosen by the library"),
                      "batched": batched, "l2": "flushed between timed steps (512 MB write)",
                      "ranks": "one independent set of instances per rank"},
           "gpu_launches": launches, "clocks": clocks, "roofline": roofline, "e2e": e2e,
           "stages": stage_summary(stages, args.steps) if stages else None,
           "fp64_same_target": fp64_out,
           "mixed_vs_fp64": (value / fp64_out["interactions_per_s"]) if fp64_out else None,
           "variants": var_out, "batched": batch_out,
           "alu_peaks_measured": alu}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sets = {"headline": head}
        if fp64_plans:
            sets["fp64_same_target"] = fp64_plans
        sets.update(var_plans)
        out["cpu_baseline"] = cpu_baseline(insts, q64, sets, runner, buf, dtype_of, args.cpu_seconds)
        log("cpu baseline done")
    for pls in [head] + ([fp64_plans] if fp64_plans else []) + list(var_plans.values()):
        for pl in pls:
            pl.close()
    return out


def run_batched_key(lib, torch, timed, dev, target, rank):
    """The 64 uneven instances (1e4..2e6 points, depth 3-6, p 4/6/8/10, 1-8 RHS) in one
    m2l_apply_batch, autotuned at `target`, graph-captured on the first call and replayed."""
    insts = W.c5()
    plans = [make_plan(lib, wl, "auto", "auto", target=target, timing=False) for wl in insts]
    qs, os_ = [], []
    for pl, wl in zip(plans, insts):
        dt = torch.float64 if pl.query(lib.M2L_Q_PRECISION, wl.n_rhs) == lib.M2L_PREC_FP64 else torch.float32
        q = np.concatenate([wl.multipoles(l, rng_offset=rank).reshape(-1) for l in wl.levels])
        qs.append(torch.from_numpy(q).to(dt).to(dev))
        os_.append(torch.empty_like(qs[-1]))
    hs, qp, op, rs = [pl.handle for pl in plans], [q.data_ptr() for q in qs], [o.data_ptr() for o in os_], \
        [wl.n_rhs for wl in insts]

    def run():
        rc = lib.m2l_apply_batch(hs, qp, op, rs)
        if rc != lib.M2L_OK:
            raise lib.M2LError(rc, lib.m2l_last_error())

    ms, _, _, _ = timed(run, 2, 3)
    m = sum(ms) / len(ms)
    inter = sum(pl.pairs(-1) * wl.n_rhs for pl, wl in zip(plans, insts))
    hist = {}
    for pl, wl in zip(plans, insts):
        f, p_ = resolved(lib, pl, wl.n_rhs)
        key = f"{f}-{p_}"
        hist[key] = hist.get(key, 0) + 1
    out = {"workload": DESC["c5"], "target_rel_err": target, "interactions_per_s": inter / (m / 1e3), "ms": m,
           "steps": 2, "warmup": 3, "pairs_x_rhs": int(inter), "forms": hist,
           "launches_per_pass": plans[0].query(lib.M2L_Q_LAUNCHES)}
    for pl in plans:
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
    W_root = wl_root_width(wl)
    while True:
        for l in wl.levels:
            B = wl.n_boxes(l)
            keys = None if wl.keys[l] is None else wl.keys[l].astype(np.int64)
            tg = rng.choice(B, size=min(B, 16), replace=False)
            L, phi = M.m2l_dense(wl.p, l, qs[l], keys=keys, targets=tg, root_width=W_root)
            results[l][0].append(tg)
            results[l][1].append(phi * (W_root / 2.0 ** l))   # check potential of a unit-width box
            results[l][2].append(L)
            done_pairs += int(M.interaction_csr(l, keys, tg)[2][-1])
        batches += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return done_pairs * R, el, results, batches


def cpu_baseline(insts, q64, sets, runner, buf, dtype_of, seconds):
    """The FP64 oracle on this host's cores, on a bounded sample of the workload's instances; also
    the error (Eq. 16) of every timed set of plans on the sampled targets: each set is re-run the
    way the timed loop runs it, once with check potentials and once with locals as output."""
    import torch
    from oracle import m2l as M
    cores = os.cpu_count()
    order = sorted(range(len(insts)), key=lambda i: -insts[i].n_boxes(insts[i].depth))[:4]
    budget = seconds / len(order)
    inter, el, batches = 0, 0.0, 0
    samples = {}
    for i in order:
        it, e_, res, b_ = _oracle_sample(insts[i], q64[i], budget)
        inter += it
        el += e_
        batches += b_
        samples[i] = res
    errs = {}
    for name, plans in sets.items():
        e = {"check_potential_rel_err_per_level": [], "locals_rel_err_per_level": [],
             "check_potential_max_target_rel_err": 0.0}
        outs = {i: {} for i in order}
        for mode in ("check", "locals"):
            for pl in plans:
                pl.set(output=mode)
            runner(plans)()
            torch.cuda.synchronize()
            for i in order:
                outs[i][mode] = buf(i, dtype_of(plans[i], insts[i]))[1].double().cpu().numpy()
        for pl in plans:
            pl.set(output="locals")
        for i in order:
            wl, res = insts[i], samples[i]
            n, R = W.n_surface(wl.p), wl.n_rhs
            off = 0
            for l in wl.levels:
                B = wl.n_boxes(l)
                c = outs[i]["check"][off:off + B * R * n].reshape(B, R, n)
                lo = outs[i]["locals"][off:off + B * R * n].reshape(B, R, n)
                off += B * R * n
                tg = np.concatenate(res[l][0])
                if len(tg) == 0:
                    continue
                ref = np.concatenate(res[l][1])
                e["check_potential_rel_err_per_level"].append(M.rel_l2_error(ref, c[tg]))
                e["check_potential_max_target_rel_err"] = max(e["check_potential_max_target_rel_err"],
                                                              M.max_target_rel_error(ref, c[tg]))
                e["locals_rel_err_per_level"].append(
                    M.check_norm_error(wl.p, l, np.concatenate(res[l][2]), lo[tg], root_width=wl_root_width(wl)))
        errs[name] = e
    return {"value": inter / el, "unit": UNIT, "cores": cores, "cpu": host_cpu(), "kind": "oracle",
            "sample": f"{batches} batches of up to 16 random target boxes per level of the "
                      f"{len(order)} largest instance(s), dense FP64 definition (per-pair kernel evaluation "
                      f"+ pseudo-inverse), {el:.1f} s",
            "rel_err_vs_oracle": errs}


def host_cpu():
    """Architecture and CPU model of this host, for the CPU legs' records."""
    import platform
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return f"{platform.machine()} {model}".strip()


def wl_root_width(wl):
    return 2.0 if wl.name == "c4" else 1.0


def run_reference(args):
    """The oracle (FP64, this host's cores) timed on bounded samples of the same workload."""
    insts, _, _ = workload_spec(args.workload, args.depth)
    wl = max(insts, key=lambda w: w.n_boxes(w.depth))
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
            "config": {"workload": DESC[args.workload], "levels": wl.levels, "target_rel_err": 0.0},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "cpu": host_cpu(), "kind": "oracle",
                             "sample": f"per step about {per_step:.0f} s of random target boxes (16 per level "
                                       f"per batch) of the same workload, dense FP64 definition"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_fmm(args):
    """The whole FMM (P2M, M2M, M2L, L2L, L2P, P2P; FP64) on the 1M-point cloud (depth 5, p = 6,
    M2L in the BLAS form at rank 1e-7 with directional factors at 1e-8, or the FFT form with
    --variants fft). Charges resident on the device; the plan (tree, operators) is built before
    the timed region. Accuracy: Eq. 16 against direct summation on a seeded sample of 1,000
    targets (the oracle's direct sum on this host)."""
    import torch
    from oracle import _cdirect
    from paper_2408_07436_gb300 import m2l as lib
    wl = W.c2(depth=args.depth)
    rng = np.random.default_rng(W.SEED_BASE + 2)
    pts = rng.random((wl.n_points, 3))
    q = rng.uniform(-1.0, 1.0, wl.n_points)
    form = (args.variants or "blas").split(",")[0].split("-")[0]
    fmm = lib.FMM(pts, depth=wl.depth, p=wl.p, rank_tol=wl.rank_tol if form == "blas" else 0.0)
    fmm.set_m2l(form=form, dir_tol=wl.dir_tol if form == "blas" else None)
    qd = torch.from_numpy(q).cuda()
    out = torch.empty_like(qd)
    for _ in range(args.warmup):
        fmm.evaluate(qd, out)
    torch.cuda.synchronize()
    sampler = ClockSampler()
    sampler.start()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        fmm.evaluate(qd, out)  # synchronous
    el = (time.perf_counter() - t0) / args.steps
    clocks = sampler.stop()
    pot = out.cpu().numpy()
    sample = np.sort(rng.choice(wl.n_points, 1000, replace=False))
    ref = _cdirect.direct_potential(pts[sample], pts, q)
    err = float(np.linalg.norm(pot[sample] - ref) / np.linalg.norm(ref))
    pairs = fmm.m2l_query(lib.M2L_Q_PAIRS, -1)
    fmm.close()
    return {"metric": "whole FMM potentials/s (FP64)", "value": wl.n_points / el, "unit": "points/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"laplace3d whole FMM uniform-cube {wl.n_points} points depth{wl.depth} p{wl.p} "
                                   f"m2l {form}" + (f"(rank_tol {wl.rank_tol:g}, directional {wl.dir_tol:g})"
                                                     if form == "blas" else "(grid 12^3)"),
                       "m2l_pairs": int(pairs), "timing": "wall clock around synchronous evaluations"},
            "rel_err_vs_direct_1000_targets": err, "clocks": clocks}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c2", "c3", "c4", "c5", "fmm"],
                    help="c3 (default): the 8M-point, p = 8 workload; c2: 1M points, p = 6; c4: sphere surface, "
                         "32 RHS; c5: 64 uneven instances batched; fmm: the whole FMM on the 1M-point cloud")
    ap.add_argument("--target", type=float, default=DEFAULT_TARGET,
                    help="relative error (Eq. 16) the headline and the FP64 comparison must meet")
    ap.add_argument("--variants", default=None, help="comma list of form-precision timed beside the headline "
                                                     "(default: the workload's; empty: none)")
    ap.add_argument("--headline", default=None, help="form-precision of the headline instead of the autotuner's "
                    "choice at the target (e.g. fft-tf32x3; for profiling runs, whose timings mislead the tuner)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison at the same target")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched 64-instance key")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-seconds", type=float, default=6.0)
    ap.add_argument("--depth", type=int, default=5, help="tree depth of the 1M-point workload (c2, fmm)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    if args.workload == "fmm":
        if rank == 0:
            print(json.dumps(run_fmm(args)))
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
