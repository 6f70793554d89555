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

VARIANTS = ["blas-fp64", "blas-fp32", "blas-tf32x3", "blas-bf16x3", "fft-fp64", "fft-fp32"]
METRIC = "M2L interactions/s and % roofline: mixed+batched vs FP64 GPU at stated rel err"
UNIT = "interactions/s"
WORKLOAD = ("laplace3d-m2l uniform-cube 1M points depth5 p6 1rhs blas(rank_tol 1e-7, directional 1e-8)+fft(grid 11^3) "
            "fp64+fp32+tf32x3+bf16x3")

# Nominal per-GPU figures (GB300) used where no measured peak exists.
NOMINAL_FP64_TFLOPS = 1.25       # FP64 (vector and tensor) dense
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a workload's dominant
# kernel from one ncu capture, with the SHA-256 of the source file the kernel was built from; the
# summary and command are in profiles/. A source that has changed since reports null.
TRAFFIC = {
    ("c2", 5, "blas-fp64:contract"): {"bytes": 139138560 + 33806592,
                                        "source": "paper_2408_07436_gb300/csrc/kernels_simt.cu",
                                        "sha256": "50642335be9d49633f0d86f1977242f8d8c5ed997eb7bda25b42405aba4c86d0"},
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


def workload_spec(name, depth):
    """(instances, variants, batched, target_tol, description) of a named workload."""
    if name == "c2":
        return [W.c2(depth=depth)], VARIANTS, False, None, WORKLOAD
    if name == "c3":
        return ([W.c3()], ["blas-bf16x3", "blas-tf32x3", "blas-fp64", "fft-fp32", "fft-fp64"], False, None,
                "laplace3d-m2l uniform-cube 8M points depth6 p8 1rhs blas(rank_tol 1e-7, directional 1e-8) bf16x3/tf32x3/fp64 + fft fp32/fp64")
    if name == "c4":
        return ([W.c4()], ["blas-bf16x3", "blas-tf32x3", "fft-fp32"], False, None,
                "laplace3d-m2l unit-sphere-surface 2M points depth6 p6 32rhs pruned boxes blas(rank_tol 1e-7) bf16x3/tf32x3 + fft fp32")
    if name == "c5":
        return (W.c5(), ["auto-auto"], True, 1e-6,
                "laplace3d-m2l 64 uneven instances (1e4..2e6 points, depth 3-6, p 4/6/8/10, 1-8 rhs) one batched "
                "graph-replayed pass, autotuned form/precision at 1e-6")
    raise ValueError(name)


def log(msg):
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2408_07436_gb300 import m2l as lib

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    insts, variants, batched, target_tol, desc = workload_spec(args.workload, args.depth)
    if args.variants:
        variants = args.variants.split(",")
    # every rank draws its own independent instances of the workload
    q64 = [np.concatenate([wl.multipoles(l, rng_offset=rank).reshape(-1) for l in wl.levels]) for wl in insts]
    plans = {v: [] for v in variants}
    bufs = {}       # (instance, dtype) -> (q, out)
    dtypes = {}     # (variant, instance) -> dtype
    for v in variants:
        form, prec = variant_parts(v)
        for i, wl in enumerate(insts):
            tol = wl.rank_tol if form in ("blas", "auto") else 0.0
            pl = lib.Plan(wl.depth, wl.p, tol, form=form, precision=prec).set(timing=0 if batched else 1)
            if form == "fft" and wl.fft_grid:
                pl.set(fft_grid=wl.fft_grid)
            if form == "blas" and prec in ("fp64", "fp32") and wl.dir_tol:
                pl.set(dir_tol=wl.dir_tol)  # the CUDA-core contraction applies Eq. 15's factors
            if target_tol is not None:
                pl.set(target_tol=target_tol)
            for l in wl.levels:
                if wl.keys[l] is not None:
                    pl.set_boxes(l, wl.keys[l])
            pl.set_stream()
            plans[v].append(pl)
            pr = pl.query(lib.M2L_Q_PRECISION, wl.n_rhs)
            dt = torch.float64 if pr == lib.M2L_PREC_FP64 else torch.float32
            dtypes[(v, i)] = dt
            if (i, dt) not in bufs:
                bufs[(i, dt)] = (torch.from_numpy(q64[i]).to(dt).to(dev), torch.empty(len(q64[i]), dtype=dt, device=dev))
    log(f"{len(insts)} instance(s), {len(variants)} variant(s): plans ready")
    pairs = [plans[variants[0]][i].pairs(-1) for i in range(len(insts))]
    inter_variant = sum(pairs[i] * insts[i].n_rhs for i in range(len(insts)))
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def run_variant(v):
        if batched:
            qs = [bufs[(i, dtypes[(v, i)])][0] for i in range(len(insts))]
            os_ = [bufs[(i, dtypes[(v, i)])][1] for i in range(len(insts))]
            rc = lib.m2l_apply_batch([pl.handle for pl in plans[v]], [q.data_ptr() for q in qs],
                                     [o.data_ptr() for o in os_], [wl.n_rhs for wl in insts])
            if rc != lib.M2L_OK:
                raise lib.M2LError(rc, lib.m2l_last_error())
        else:
            for i, wl in enumerate(insts):
                qd, od = bufs[(i, dtypes[(v, i)])]
                plans[v][i].apply(qd, od, -1, wl.n_rhs)

    for _ in range(args.warmup):
        for v in variants:
            run_variant(v)
    torch.cuda.synchronize()
    log("warm-up done")
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
        for j, v in enumerate(variants):
            run_variant(v)
            evs[j + 1].record(stream)
        torch.cuda.synchronize()
        total_ms += evs[0].elapsed_time(evs[-1])
        for j, v in enumerate(variants):
            var_ms[v] += evs[j].elapsed_time(evs[j + 1])
            if batched:
                launches += plans[v][0].query(lib.M2L_Q_LAUNCHES)
                continue
            for pl in plans[v]:
                for name, (ms, nl) in pl.stage_times().items():
                    a = stage_acc[v].setdefault(name, [0.0, 0])
                    a[0] += ms
                    a[1] += nl
                    launches += nl
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = sampler.stop()
    log(f"timed steps done: {total_ms / args.steps:.1f} ms per step")
    ms_step = total_ms / args.steps
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms_step], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    inter_step = inter_variant * len(variants)
    value = world * inter_step / (ms_step / 1e3)
    steps_for_stages = args.steps
    if batched:
        # stage times of a batch: one separate, untimed apply of the largest instance on a fresh plan
        big = max(range(len(insts)), key=lambda i: pairs[i] * insts[i].n_rhs)
        wl = insts[big]
        for v in variants:
            src = plans[v][big]
            f = src.query(lib.M2L_Q_FORM, wl.n_rhs)
            pr = src.query(lib.M2L_Q_PRECISION, wl.n_rhs)
            fname = "blas" if f == lib.M2L_FORM_BLAS else "fft"
            pname = {lib.M2L_PREC_FP64: "fp64", lib.M2L_PREC_FP32: "fp32", lib.M2L_PREC_TF32X3: "tf32x3",
                     lib.M2L_PREC_BF16X3: "bf16x3"}[pr]
            probe = lib.Plan(wl.depth, wl.p, wl.rank_tol if fname == "blas" else 0.0, form=fname,
                             precision=pname).set(timing=1)
            for l in wl.levels:
                if wl.keys[l] is not None:
                    probe.set_boxes(l, wl.keys[l])
            probe.set_stream()
            qd, od = bufs[(big, dtypes[(v, big)])]
            probe.apply(qd, od, -1, wl.n_rhs)
            for name, (ms, nl) in probe.stage_times().items():
                a = stage_acc[v].setdefault(name, [0.0, 0])
                a[0] += ms
                a[1] += nl
            probe_work = algorithmic_work(probe, fname, pname, wl.n_rhs)
            stage_acc[v]["_algorithmic"] = probe_work
            stage_acc[v]["_prec"] = pname
            probe.close()
        steps_for_stages = 1

    # roofline of the dominant kernel of each variant and of the step
    peaks = measured_peaks()

    def peak_for(prec):
        if prec == "fp64":
            return NOMINAL_FP64_TFLOPS, "alu", "nominal GB300 FP64 1.25 TFLOP/s"
        if prec == "fp32":
            return fp32_alu_peak_tflops(), "alu", "152 SM x 128 FP32 lanes x 2 flops x 2070 MHz"
        bf = peaks.get("bf16_tflops_sustained", 1700.0)
        if prec == "bf16x3":
            return bf / 3.0, "tensor", "of measured: bf16 sustained / 3 (each useful product is 3 MMAs)"
        return bf / 2.0 / 3.0, "tensor", "of measured: bf16 sustained / 2 (nominal tf32 ratio) / 3 (3 MMAs per product)"

    var_out = {}
    best = None
    for v in variants:
        # algorithmic work per stage, summed over instances (each resolved to its own precision);
        # for a batch, the stage times and work are those of its largest instance
        probe_work = stage_acc[v].pop("_algorithmic", None)
        probe_prec = stage_acc[v].pop("_prec", None)
        work, prec_of = {}, None
        for i, (pl, wl) in enumerate(zip(plans[v], insts)):
            f = pl.query(lib.M2L_Q_FORM, wl.n_rhs)
            pr = pl.query(lib.M2L_Q_PRECISION, wl.n_rhs)
            fname = "blas" if f == lib.M2L_FORM_BLAS else "fft"
            pname = {lib.M2L_PREC_FP64: "fp64", lib.M2L_PREC_FP32: "fp32", lib.M2L_PREC_TF32X3: "tf32x3",
                     lib.M2L_PREC_BF16X3: "bf16x3"}[pr]
            prec_of = pname if prec_of in (None, pname) else "mixed"
            for k, w in algorithmic_work(pl, fname, pname, wl.n_rhs).items():
                work[k] = work.get(k, 0.0) + w
        prec_all = prec_of
        if probe_work is not None:
            work, prec_of = probe_work, probe_prec
        stages = {}
        for name, (ms, nl) in stage_acc[v].items():
            if nl == 0:
                continue
            per_launch_ms = ms / nl
            flops_launch = work.get(name, 0.0) * steps_for_stages / nl
            stages[name] = {"ms_per_step": ms / steps_for_stages, "launches_per_step": nl / steps_for_stages,
                            "gflops": flops_launch / (per_launch_ms / 1e3) / 1e9 if per_launch_ms > 0 else None}
        var_out[v] = {"interactions_per_s": inter_variant / (var_ms[v] / args.steps / 1e3), "ms": var_ms[v] / args.steps,
                      "stages": stages, "precision": prec_all}
        if probe_work is not None:
            var_out[v]["stages_of"] = "largest instance, separate apply"
        if insts and variant_parts(v)[0] == "blas":
            var_out[v]["rank"] = [pl.query(lib.M2L_Q_RANK) for pl in plans[v]][:4]
        if stages and prec_of != "mixed":
            name = max(stages, key=lambda n: stages[n]["ms_per_step"])
            ms_tot, nl = stage_acc[v][name]
            pk, bound, note = peak_for(prec_of)
            per_launch_ms = ms_tot / nl
            ach = work.get(name, 0.0) * steps_for_stages / nl / (per_launch_ms / 1e3) / 1e12
            rf = {"bound": bound, "kernel": f"{v}:{name}", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                  "frac": ach / pk, "traffic": measured_traffic(args.workload, args.depth, f"{v}:{name}"),
                  "peak_source": note}
            var_out[v]["roofline"] = rf
            if best is None or ms_tot > best[0]:
                best = (ms_tot, rf)
    roofline = best[1] if best else None

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        hq = {k: bufs[k][0].cpu().pin_memory() for k in bufs}
        ho = {k: torch.empty_like(hq[k]).pin_memory() for k in bufs}

        def e2e_pass():
            for v in variants:
                if batched:
                    for i in range(len(insts)):
                        k = (i, dtypes[(v, i)])
                        bufs[k][0].copy_(hq[k], non_blocking=True)
                    run_variant(v)
                    for i in range(len(insts)):
                        k = (i, dtypes[(v, i)])
                        ho[k].copy_(bufs[k][1], non_blocking=True)
                    torch.cuda.synchronize()
                else:
                    for i, wl in enumerate(insts):
                        k = (i, dtypes[(v, i)])
                        plans[v][i].apply(hq[k], ho[k], -1, wl.n_rhs)

        e2e_pass()  # warm the staging buffers
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_pass()
        el = time.perf_counter() - t0
        h2d = sum(hq[(i, dtypes[(v, i)])].numel() * hq[(i, dtypes[(v, i)])].element_size()
                  for v in variants for i in range(len(insts)))
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([el], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        e2e = {"value": world * inter_step * args.steps / el, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": h2d}

    mixed = [v for v in variants if var_out[v].get("precision") in ("tf32x3", "bf16x3", "fp32")]
    fp64 = [v for v in variants if var_out[v].get("precision") == "fp64"]
    headline = None
    if mixed and fp64:
        bm = max(mixed, key=lambda v: var_out[v]["interactions_per_s"])
        bf = max(fp64, key=lambda v: var_out[v]["interactions_per_s"])
        headline = {"fastest_reduced_precision": bm, "fastest_fp64": bf,
                    "speedup": var_out[bm]["interactions_per_s"] / var_out[bf]["interactions_per_s"]}
    precs = sorted({var_out[v].get("precision") or "?" for v in variants})
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "+".join(precs), "data": "synthetic",
           "config": {"workload": desc, "instances": len(insts), "pairs_per_variant": int(sum(pairs)),
                      "interactions_per_variant": int(inter_variant), "variants": variants,
                      "batched": batched, "target_tol": target_tol,
                      "l2": "flushed between timed steps (512 MB write)",
                      "ranks": "one independent set of instances per rank"},
           "gpu_launches": launches, "clocks": clocks, "roofline": roofline, "e2e": e2e, "variants": var_out,
           "mixed_vs_fp64": headline}
    log("e2e done")
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(insts, q64, plans, bufs, dtypes, args.cpu_seconds, run_variant)
        log("cpu baseline done")
    for v in variants:
        for pl in plans[v]:
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


def cpu_baseline(insts, q64, plans, bufs, dtypes, seconds, run_variant):
    """The FP64 oracle on this host's cores, on a bounded sample of the workload's instances; also
    the error of each variant on the sampled targets (Eq. 16). Each variant is re-run the way the
    timed loop runs it (`run_variant`: one batch call for a batched workload), once with check
    potentials and once with locals as output."""
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
    errs = {v: {"check_potential_rel_err_per_level": [], "locals_rel_err_per_level": []} for v in plans}
    for v in plans:
        outs = {i: {} for i in order}
        for mode in ("check", "locals"):
            for pl in plans[v]:
                pl.set(output=mode)
            run_variant(v)
            torch.cuda.synchronize()
            for i in order:
                outs[i][mode] = bufs[(i, dtypes[(v, i)])][1].double().cpu().numpy()
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
                errs[v]["check_potential_rel_err_per_level"].append(M.rel_l2_error(np.concatenate(res[l][1]), c[tg]))
                errs[v]["locals_rel_err_per_level"].append(
                    M.check_norm_error(wl.p, l, np.concatenate(res[l][2]), lo[tg], root_width=wl_root_width(wl)))
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
    insts, _, _, _, desc = workload_spec(args.workload, args.depth)
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
            "config": {"workload": desc, "levels": wl.levels},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "cpu": host_cpu(), "kind": "oracle",
                             "sample": f"per step about {per_step:.0f} s of random target boxes (16 per level "
                                       f"per batch) of the same workload, dense FP64 definition"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_fmm(args):
    """The whole FMM (P2M, M2M, M2L, L2L, L2P, P2P; FP64) on the 1M-point cloud of the default
    workload (depth 5, p = 6, M2L in the BLAS form at rank 1e-7 with directional factors at 1e-8,
    or the FFT form with --variants fft). Charges resident on the device; the plan (tree,
    operators) is built before the timed region. Accuracy: Eq. 16 against direct summation on a
    seeded sample of 1,000 targets (the oracle's direct sum on this host)."""
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
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c4", "c5", "fmm"],
                    help="c2 (default): the 1M-point workload; c3/c4/c5: precision, RHS-batching and instance-batching "
                         "studies; fmm: the whole FMM around M2L on the 1M-point cloud")
    ap.add_argument("--variants", default=None, help="comma list of form-precision (default: the workload's)")
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
