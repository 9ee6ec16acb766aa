"""Benchmark: curve points evaluated per second per evaluator, as a speed-up
over FP32 Horner on the same GPU, with the max normalised error against the
FP64 oracle.

Default workload (precision/texture), one step = one bez_eval call over
1,048,576 cubic 3D Bezier curves (control points U[-1,1]^3 FP32), each at
1024 parameters drawn U[0,1) inside the kernel, reduced to one polyline
length per curve (no point stores): per-curve setup, parameter draw,
evaluation and warp-shuffle reduction in one kernel (texture variants add
the atlas packing kernel).  The same line reports the C0 chain part of the
workload (16,384 chains x 64 quadratic segments, 65,536 parameters each,
register de Casteljau vs the zig-zag texture).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload all|precision|plain|chains|batch|tensor|fit]

Prints one JSON line.  The default (all) line is the precision workload's
headline, and on one GPU its "configs" object adds the other four
workloads (plain, batch, tensor, fit), each with its own throughput,
roofline, accuracy against the oracle and clock sample.  Under torchrun
(N > 1) every rank evaluates its own precision batch of the same size (weak
scaling, different seeds); the only cross-rank traffic is the timing barrier
and a max over ranks of the timed duration.  --workload X prints the line
of one workload alone.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "curve points evaluated/sec vs FP32 Horner on same GB300, at max err vs FP64 oracle"
N_CURVES = 1 << 20
N_T = 1024


def workload_name(n_curves=N_CURVES, n_t=N_T):
    return (f"precision/texture: {n_curves:,} cubic 3D Bezier curves (U[-1,1]^3 FP32), {n_t} parameters per curve "
            "drawn U[0,1) in-kernel, fused per-curve polyline length (no point stores)")

# Algorithmic lane operations per point (cubic, 3D):
# parameter draw 9 (xor of the sample index into the curve key, whose first
# lowbias32 shift-xor is applied once per curve since the index is < 2^16;
# 2 mul + 2 shift + 2 xor; funnel shift; subtract) + evaluation + polyline
# step 8 (3 sub, mul + 2 fma, sqrt, add).  The centred form folds its shift by
# 1/2 into the draw's subtraction, so it evaluates in 9 fma like Horner.
T_OPS, LEN_OPS = 9, 8

# DRAM bytes (read + write) per launch from one ncu capture of the current
# kernels, per unit of work; null in the JSON line for other kernels.  The
# curve kernel was captured on 131,072 curves (6,307,584 B: the control
# points; the 4 B lengths stay in L2) and scales with the curve count; the
# surface kernel on the full 65,536-patch tensor workload; the fused adjoint
# on the full 65,536 x 512 fit step.
TRAFFIC_PER_CURVE = {"HORNER_CENTRED": 6312448 / 131072}
# the kernel behind each headline variant's fused length (cubic 3D, hashed t)
KERNEL_NAME = {"HORNER_CENTRED": "k_curve_group<3, 4> (four lanes per curve)", "HALF2": "k_curve_h2"}
TRAFFIC_SURFACE_65536 = 12652544 + 742988544
TRAFFIC_FIT_65536x512 = 540180736 + 121996800
EVAL_OPS = {"HORNER": 9, "HORNER_CENTRED": 9, "HALF2": 5, "BERNSTEIN": 19, "SEILER": 16, "DECASTELJAU": 36,
            "TEX_DECASTELJAU": 3, "TEX_SEILER": 3, "TEX_HYBRID": 10, "TEX_SEILER_S8": 3, "TEX_SEILER_S4": 3}
# filtered fetches per point and the peak they are held to
TEX_FETCHES = {"TEX_DECASTELJAU": (1, "tex3d_f32"), "TEX_SEILER": (1, "tex2d_f32"), "TEX_HYBRID": (2, "tex2d_f32"),
               "TEX_SEILER_S8": (1, "tex2d_f32"), "TEX_SEILER_S4": (1, "tex2d_f32")}
REG_VARIANTS = ["HORNER", "HORNER_CENTRED", "BERNSTEIN", "SEILER", "DECASTELJAU", "HALF2"]
TEX_VARIANTS = ["TEX_DECASTELJAU", "TEX_SEILER", "TEX_HYBRID", "TEX_SEILER_S8", "TEX_SEILER_S4"]
VARIANTS = REG_VARIANTS + TEX_VARIANTS
# bench name -> (bez_variant name, tex_spread): TEX_SEILER_S8 / _S4 are the
# cubic Seiler tile spread over 9 x 9 / 5 x 5 texels
VARIANT_SPEC = {v: (v, 0) for v in VARIANTS}
VARIANT_SPEC["TEX_SEILER_S8"] = ("TEX_SEILER", 8)
VARIANT_SPEC["TEX_SEILER_S4"] = ("TEX_SEILER", 4)
FP32_BAR, TEX_BAR = 1e-6, 2e-3
FALLBACK_SMS, LANES = 152, 128


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return None


def sm_count(dev=0):
    """Streaming multiprocessors of the device (None without a GPU)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.get_device_properties(dev).multi_processor_count)
    except Exception:  # pragma: no cover - no torch / no device
        pass
    return None


def alu_peak(peaks, sms=None):
    """FP32/INT32 lane-operation issue peak: SMs x 128 lanes x max clock,
    with the SM count read from the device (152 when none is given)."""
    mhz = float(peaks.get("sm_max_mhz", 2070.0)) if peaks else 2070.0
    src = "device" if sms else "fallback"
    sms = sms or FALLBACK_SMS
    return sms * LANES * mhz * 1e6, f"derived: {sms} SMs ({src}) x {LANES} lanes x {mhz:.0f} MHz"


def hbm_peak(peaks):
    if peaks and "hbm_gbs" in peaks:
        return float(peaks["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs, copy)"
    return 6800.0, "of fallback (6.8 TB/s)"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # nvidia-smi takes a moment to start: let its first sample arrive
            # before the measured work begins, so short workloads are covered
            t0 = time.perf_counter()
            while not self.lines and self.proc.poll() is None and time.perf_counter() - t0 < 3.0:
                time.sleep(0.01)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


class Timer:
    """Times K steps with CUDA events on the current stream, flushing L2
    (256 MiB device write) before each step outside the timed region; the
    library's own events bracket its main kernels."""

    def __init__(self, torch, ctx, dev, world):
        self.torch, self.ctx, self.dev, self.world = torch, ctx, dev, world
        self.flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        self.stream = torch.cuda.current_stream(dev)

    def run(self, step, steps, warmup):
        torch = self.torch
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()
        self.ctx.reset_stats()
        self.ctx.set_timing(True)
        evs = []
        torch.cuda.synchronize()
        for _ in range(steps):
            self.flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(self.stream)
            step()
            b.record(self.stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()
        self.ctx.set_timing(False)
        st = self.ctx.stats()
        return sum(a.elapsed_time(b) for a, b in evs), st


def max_over_ranks(torch, dev, world, ms):
    if world == 1:
        return ms
    import torch.distributed as dist
    t = torch.tensor([ms], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measure_peaks(bez, ctx):
    out = {}
    for k in ("fma", "tex2d_f32", "tex2d_f16", "tex3d_f32", "tex3d_f16"):
        out[k] = bez.bez_measure_peak(k, ctx=ctx)
    return out


# ------------------------------------------------------------------ default workload

def run_precision(args, rank, world, local_rank):
    import torch

    from paper_2603_15447_gb300 import bez, synth

    dev = torch.device("cuda", local_rank)
    seed = synth.BASE_SEED + 1 + 1000 * rank
    ctrl_np = synth.precision(seed=seed, n_curves=args.n_curves)
    ctrl = torch.from_numpy(ctrl_np).to(dev)
    out = torch.empty(args.n_curves, dtype=torch.float32, device=dev)
    ctx = bez.context(local_rank)
    timer = Timer(torch, ctx, dev, world)
    ts = synth.PRECISION_T_STREAM

    def step_for(v, c=ctrl, fmt=bez.TexFormat.AUTO):
        var, spread = VARIANT_SPEC[v]

        def step():
            bez.bez_eval(c, None, n_t=args.n_t, variant=bez.Variant[var], out_mode=bez.OutMode.POLYLINE_LENGTH,
                         t_mode=bez.TMode.HASH, seed=seed, stream_id=ts, out=out, ctx=ctx, tex_format=fmt,
                         tex_spread=spread)
        return step

    run_variants = [v for v in VARIANTS if v in args.variants.split(",")] if args.variants else list(VARIANTS)
    for must in ("HORNER", args.variant):
        if must not in run_variants:
            run_variants.append(must)
    results = {}
    results16 = {}
    ctrl16 = None if args.skip_f16 else ctrl.half()
    with ClockSampler(local_rank) as clocks:
        for v in run_variants:
            ms, st = timer.run(step_for(v), args.steps, args.warmup)
            results[v] = {"ms": ms, "stats": st}
        if ctrl16 is not None:
            # half storage (half4 texture atlases), FP32 arithmetic
            for v in run_variants:
                ms, st = timer.run(step_for(v, ctrl16), args.steps, args.warmup)
                results16[v] = {"ms": ms, "stats": st}
            # bfloat16 storage, FP32 arithmetic (register evaluators: no bfloat16 texel format)
            results_bf = {}
            ctrl_bf = ctrl.bfloat16()
            for v in run_variants:
                if v in REG_VARIANTS and v != "HALF2":
                    ms, st = timer.run(step_for(v, ctrl_bf), args.steps, args.warmup)
                    results_bf[v] = {"ms": ms, "stats": st}
        # unorm texels with per-curve rescale (texture variants only)
        results_unorm = {}
        if not args.skip_f16:
            for fmt in (bez.TexFormat.UNORM16, bez.TexFormat.UNORM8):
                for v in run_variants:
                    if v in TEX_FETCHES:
                        ms, st = timer.run(step_for(v, ctrl, fmt), args.steps, args.warmup)
                        results_unorm[(fmt.name, v)] = {"ms": ms, "stats": st}
        # co-issue: `share` of every 8 samples through the texture unit, the
        # rest on the FP32 pipes, in one kernel
        coissue = {}
        if not args.skip_coissue:
            for label, c in (("f32", ctrl), ("f16", ctrl16)):
                if c is None:
                    continue
                for share in range(1, 8):
                    def cstep(c=c, share=share):
                        bez.bez_eval(c, None, n_t=args.n_t, variant=bez.Variant.COISSUE,
                                     out_mode=bez.OutMode.POLYLINE_LENGTH, t_mode=bez.TMode.HASH, seed=seed,
                                     stream_id=ts, out=out, ctx=ctx, tex_share=share)
                    ms, st = timer.run(cstep, args.steps, args.warmup)
                    coissue[f"{label}_share{share}of8"] = {
                        "points_per_s": args.n_curves * args.n_t * args.steps / (ms * 1e-3),
                        "kernel_ms": st["timed_ms"] / max(st["timed_launches"], 1)}
    clock_summary = clocks.summary()

    # chain part of the workload: register de Casteljau and centred Horner vs zig-zag texture
    chains = None
    if not args.skip_chains:
        cctrl_np, _ = synth.chains(n_chains=args.n_chains, n_t=1)
        cctrl = torch.from_numpy(cctrl_np).to(dev)
        cout = torch.empty(args.n_chains, dtype=torch.float32, device=dev)
        chains = {}
        csteps = max(args.steps // 4, 3)
        # name -> (variant, tex_spread, texel format)
        chain_variants = {"DECASTELJAU": ("DECASTELJAU", 0, "AUTO"), "HORNER_CENTRED": ("HORNER_CENTRED", 0, "AUTO"),
                          "TEX_DECASTELJAU": ("TEX_DECASTELJAU", 0, "AUTO"),
                          "TEX_DECASTELJAU_S4": ("TEX_DECASTELJAU", 4, "AUTO"),
                          "TEX_DECASTELJAU_S4_UNORM16": ("TEX_DECASTELJAU", 4, "UNORM16")}
        for name, (v, spread, fmt) in chain_variants.items():
            def cstep(v=v, spread=spread, fmt=fmt, o=cout, n_t=args.chain_t, c=cctrl):
                bez.bez_eval_piecewise(c, 64, 2, None, n_t=n_t, variant=bez.Variant[v],
                                       out_mode=bez.OutMode.POLYLINE_LENGTH, t_mode=bez.TMode.HASH, seed=seed,
                                       stream_id=12, out=o, ctx=ctx, tex_spread=spread,
                                       tex_format=bez.TexFormat[fmt])
            ms, st = timer.run(cstep, csteps, 2)
            n_pts = args.n_chains * args.chain_t * csteps
            chains[name] = {"points_per_s": n_pts / (ms * 1e-3),
                            "kernel_ms": st["timed_ms"] / max(st["timed_launches"], 1)}
            if spread:
                chains[name]["tex_spread"] = spread
            if fmt != "AUTO":
                chains[name]["tex_format"] = fmt
        if not args.skip_accuracy:
            # points of the first chains at 4096 of their hashed parameters against the oracle
            import oracle
            nc, nt = 256, 4096
            u = oracle.hash_t(seed, 12, 0, nc, nt)
            tch = (np.float32(64) * u.astype(np.float32)).astype(np.float32)
            cref = oracle.chain(cctrl_np[:nc], 64, 2, tch)
            cdiag = np.maximum(np.linalg.norm(cref.max(axis=1) - cref.min(axis=1), axis=-1), 2.0 ** -4)
            for name, (v, spread, fmt) in chain_variants.items():
                pts = bez.bez_eval_piecewise(cctrl[:nc].contiguous(), 64, 2, None, n_t=nt, variant=bez.Variant[v],
                                             t_mode=bez.TMode.HASH, seed=seed, stream_id=12, ctx=ctx,
                                             tex_spread=spread, tex_format=bez.TexFormat[fmt])
                err = np.linalg.norm(pts.cpu().numpy().astype(np.float64) - cref, axis=-1).max(axis=1) / cdiag
                bar = TEX_BAR if v.startswith("TEX") else FP32_BAR
                chains[name].update({"max_norm_err": float(err.max()), "bar": bar,
                                     "meets_bar": bool(err.max() <= bar)})

    ms_head = max_over_ranks(torch, dev, world, results[args.variant]["ms"])

    # error of the timed kernel's own output: the headline step once more over
    # the whole batch, then the lengths of 8 blocks of 512 curves spread over
    # it (the last block ends at the last curve) against the oracle's
    length_err = None
    if not args.skip_accuracy:
        import oracle
        step_for(args.variant)()
        torch.cuda.synchronize()
        got_len = out.cpu().numpy().astype(np.float64)
        bs = min(512, args.n_curves)
        starts = np.unique(np.linspace(0, args.n_curves - bs, 8).astype(np.int64))
        rel = []
        for s0 in starts:
            Lr = oracle.hashed_bezier_polyline_length(ctrl_np[s0:s0 + bs], args.n_t, seed, ts, c0=int(s0))
            rel.append(np.abs(got_len[s0:s0 + bs] - Lr) / Lr)
        length_err = {"max_rel_length_err": float(np.max(rel)),
                      "sample": f"{len(starts)} blocks of {bs} curves spread over the batch (last block ends at "
                                f"curve {args.n_curves - 1}), lengths of the timed launch shape"}

    # end to end through the public API with pinned host buffers
    ctrl_host = torch.from_numpy(ctrl_np).pin_memory()
    out_host = torch.empty(args.n_curves, dtype=torch.float32).pin_memory()

    def e2e_step():
        bez.bez_eval(ctrl_host, None, n_t=args.n_t, variant=bez.Variant[args.variant],
                     out_mode=bez.OutMode.POLYLINE_LENGTH, t_mode=bez.TMode.HASH, seed=seed, stream_id=ts,
                     out=out_host, ctx=ctx)

    for _ in range(max(args.warmup, 1)):
        e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e2e_s = (time.perf_counter() - t0) / args.steps

    if rank != 0:
        return None
    peak_alu, peak_note = alu_peak(load_peaks(), sm_count(local_rank))
    peaks = measure_peaks(bez, ctx)
    pts_step = args.n_curves * args.n_t
    variants = {}
    for v in run_variants:
        r = results[v]
        st = r["stats"]
        kern_ms = st["timed_ms"] / max(st["timed_launches"], 1)
        ops = (T_OPS + EVAL_OPS[v] + LEN_OPS) * pts_step
        row = {"points_per_s": pts_step * args.steps / (r["ms"] * 1e-3), "ms_per_step": r["ms"] / args.steps,
               "kernel_ms": kern_ms, "ops_per_point": T_OPS + EVAL_OPS[v] + LEN_OPS,
               "alu_frac": ops / (kern_ms * 1e-3) / peak_alu}
        if v in TEX_FETCHES:
            nf, kind = TEX_FETCHES[v]
            row["fetches_per_s"] = nf * pts_step / (kern_ms * 1e-3)
            row["tex_frac"] = row["fetches_per_s"] / peaks[kind]
            row["tex_peak"] = kind
            # the step is pack + evaluate; the library's events bracket the evaluation only
            row["pack_ms"] = r["ms"] / args.steps - kern_ms
        variants[v] = row
    horner = variants["HORNER"]["points_per_s"]
    for v in run_variants:
        variants[v]["speedup_vs_horner"] = variants[v]["points_per_s"] / horner
    variants_unorm = {}
    for (fname, v), r in results_unorm.items():
        st = r["stats"]
        kern_ms = st["timed_ms"] / max(st["timed_launches"], 1)
        variants_unorm.setdefault(fname, {})[v] = {"points_per_s": pts_step * args.steps / (r["ms"] * 1e-3),
                                                   "kernel_ms": kern_ms}
    variants_bf = {}
    for v, r in (results_bf.items() if ctrl16 is not None else []):
        st = r["stats"]
        kern_ms = st["timed_ms"] / max(st["timed_launches"], 1)
        variants_bf[v] = {"points_per_s": pts_step * args.steps / (r["ms"] * 1e-3), "kernel_ms": kern_ms,
                          "speedup_vs_horner": pts_step * args.steps / (r["ms"] * 1e-3) / horner}
    variants16 = {}
    for v, r in results16.items():
        st = r["stats"]
        kern_ms = st["timed_ms"] / max(st["timed_launches"], 1)
        row = {"points_per_s": pts_step * args.steps / (r["ms"] * 1e-3), "kernel_ms": kern_ms}
        row["speedup_vs_horner"] = row["points_per_s"] / horner
        if v in TEX_FETCHES:
            nf, kind = TEX_FETCHES[v]
            kind = kind.replace("f32", "f16")
            row["fetches_per_s"] = nf * pts_step / (kern_ms * 1e-3)
            row["tex_frac"] = row["fetches_per_s"] / peaks[kind]
            row["tex_peak"] = kind
        variants16[v] = row

    if not args.skip_accuracy:
        import oracle
        ns = args.accuracy_curves
        sample = ctrl[:ns].contiguous()
        th = oracle.hash_t(seed, ts, 0, ns, args.n_t)
        ref = oracle.bezier(ctrl_np[:ns], th)
        diag = np.maximum(np.linalg.norm(ref.max(axis=1) - ref.min(axis=1), axis=-1), 2.0 ** -4)
        for v in run_variants:
            var, spread = VARIANT_SPEC[v]
            pts = bez.bez_eval(sample, None, n_t=args.n_t, variant=bez.Variant[var], t_mode=bez.TMode.HASH,
                               seed=seed, stream_id=ts, ctx=ctx, tex_spread=spread)
            err = np.linalg.norm(pts.cpu().numpy().astype(np.float64) - ref, axis=-1).max(axis=1) / diag
            bar = TEX_BAR if (v in TEX_FETCHES or v == "HALF2") else FP32_BAR
            variants[v]["max_norm_err"] = float(err.max())
            variants[v]["bar"] = bar
            variants[v]["meets_bar"] = bool(err.max() <= bar)
            for fname, tab in variants_unorm.items():
                if v in tab:
                    pts = bez.bez_eval(sample, None, n_t=args.n_t, variant=bez.Variant[var], t_mode=bez.TMode.HASH,
                                       seed=seed, stream_id=ts, ctx=ctx, tex_format=bez.TexFormat[fname],
                                       tex_spread=spread)
                    err = np.linalg.norm(pts.cpu().numpy().astype(np.float64) - ref, axis=-1).max(axis=1) / diag
                    tab[v]["max_norm_err"] = float(err.max())
            if v in variants_bf:
                # against the oracle of the FP32 control points: includes the 2^-8 storage rounding
                pts = bez.bez_eval(sample.bfloat16(), None, n_t=args.n_t, variant=bez.Variant[var],
                                   t_mode=bez.TMode.HASH, seed=seed, stream_id=ts, ctx=ctx)
                err = np.linalg.norm(pts.cpu().numpy().astype(np.float64) - ref, axis=-1).max(axis=1) / diag
                variants_bf[v]["max_norm_err"] = float(err.max())
            if v in variants16:
                # against the oracle of the FP32 control points: includes the 2^-11 storage rounding
                pts = bez.bez_eval(sample.half(), None, n_t=args.n_t, variant=bez.Variant[var],
                                   t_mode=bez.TMode.HASH, seed=seed, stream_id=ts, ctx=ctx, tex_spread=spread)
                err = np.linalg.norm(pts.cpu().numpy().astype(np.float64) - ref, axis=-1).max(axis=1) / diag
                variants16[v]["max_norm_err"] = float(err.max())

    if not args.skip_accuracy and coissue:
        # lengths of the accuracy sample against the oracle's FP64 lengths
        import oracle
        ns = args.accuracy_curves
        L = oracle.hashed_bezier_polyline_length(ctrl_np[:ns], args.n_t, seed, ts)
        for key in coissue:
            c = (ctrl if key.startswith("f32") else ctrl16)[:ns].contiguous()
            share = int(key.split("share")[1][0])
            got = bez.bez_eval(c, None, n_t=args.n_t, variant=bez.Variant.COISSUE, out_mode=bez.OutMode.POLYLINE_LENGTH,
                               t_mode=bez.TMode.HASH, seed=seed, stream_id=ts, ctx=ctx, tex_share=share)
            coissue[key]["max_rel_length_err"] = float(np.max(np.abs(got.cpu().numpy() - L) / L))

    # the fastest variant meeting each accuracy bar (FP32 1e-6; FP16 / BF16 /
    # texture 2e-3), over every measured storage and texel format, as a
    # speed-up over FP32 Horner in this run
    best_by_bar = None
    if not args.skip_accuracy:
        cands = [(v, "f32", r) for v, r in variants.items()]
        cands += [(v, "f16 storage", r) for v, r in variants16.items()]
        cands += [(v, "bf16 storage", r) for v, r in variants_bf.items()]
        cands += [(v, f"{f.lower()} texels", r) for f, tab in variants_unorm.items() for v, r in tab.items()]
        best_by_bar = {}
        for label, bar in (("fp32_1e-6", FP32_BAR), ("reduced_precision_2e-3", TEX_BAR)):
            ok = [(r["points_per_s"], v, fmt, r) for v, fmt, r in cands
                  if r.get("max_norm_err") is not None and r["max_norm_err"] <= bar]
            if ok:
                pps, v, fmt, r = max(ok, key=lambda x: x[0])
                best_by_bar[label] = {"variant": v, "storage": fmt, "points_per_s": pps,
                                      "speedup_vs_horner": pps / horner, "max_norm_err": r["max_norm_err"]}
        tex_ok = [(r["points_per_s"], v, fmt, r) for v, fmt, r in cands
                  if v.startswith("TEX") and r.get("max_norm_err") is not None and r["max_norm_err"] <= TEX_BAR]
        if tex_ok:
            pps, v, fmt, r = max(tex_ok, key=lambda x: x[0])
            best_by_bar["texture_path_2e-3"] = {"variant": v, "storage": fmt, "points_per_s": pps,
                                                "speedup_vs_horner": pps / horner, "max_norm_err": r["max_norm_err"]}
    head = variants[args.variant]
    traffic = args.traffic
    if traffic is None and args.variant in TRAFFIC_PER_CURVE:
        traffic = TRAFFIC_PER_CURVE[args.variant] * args.n_curves
    kern_ms = head["kernel_ms"]
    ops_launch = head["ops_per_point"] * pts_step
    achieved = ops_launch / (kern_ms * 1e-3)
    line = {
        "metric": METRIC,
        "value": pts_step * world * args.steps / (ms_head * 1e-3),
        "unit": "points/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_head / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": workload_name(args.n_curves, args.n_t), "variant": args.variant,
                   "n_curves": args.n_curves, "n_t": args.n_t,
                   "degree": 3, "dim": 3, "l2": "flushed between timed steps (256 MiB device write)",
                   "speedup_vs_horner": head["speedup_vs_horner"],
                   "max_norm_err": head.get("max_norm_err"),
                   "max_norm_err_sample": f"first {args.accuracy_curves} curves x {args.n_t} points",
                   **(length_err or {})},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_alu / 1e12, "unit": "Tops/s",
                     "frac": achieved / peak_alu, "traffic": traffic, "peak_source": peak_note,
                     "ops_per_launch": ops_launch,
                     "kernel": KERNEL_NAME.get(args.variant, "k_curve") + " (fused draw + eval + polyline length)",
                     "measured_fma_peak_tops": peaks["fma"] / 1e12},
        "e2e": {"value": pts_step / e2e_s, "unit": "points/s",
                "h2d_bytes_per_step": int(ctrl_np.nbytes), "d2h_bytes_per_step": int(args.n_curves * 4)},
        "gpu_launches": int(results[args.variant]["stats"]["launches"]),
        "clocks": clock_summary,
        "best_by_accuracy_bar": best_by_bar,
        "variants": variants,
        "variants_f16_storage": variants16 or None,
        "variants_bf16_storage": variants_bf or None,
        "variants_unorm_texels": variants_unorm or None,
        "coissue": coissue or None,
        "peaks_measured": {"fma_tops": peaks["fma"] / 1e12,
                           **{k + "_gfetch_s": peaks[k] / 1e9 for k in peaks if k.startswith("tex")}},
    }
    if chains is not None:
        line["chains"] = {"workload": f"{args.n_chains} C0 chains x 64 quadratic segments, {args.chain_t} "
                                      "parameters per chain drawn U[0,64) in-kernel, fused polyline length",
                          "accuracy_sample": "first 256 chains x 4096 points",
                          **chains}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(ctrl_np, seed, args.n_t, args.cpu_seconds)
    return line


def cpu_baseline(ctrl_np, seed, n_t, seconds):
    """The FP64 oracle, as it stands, on the host cores: chunks of the same
    workload until about `seconds` of wall time or the whole batch is done."""
    import oracle
    from paper_2603_15447_gb300 import synth
    threads = oracle.default_threads()
    chunk = 8192
    done = 0
    t0 = time.perf_counter()
    while done < ctrl_np.shape[0] and time.perf_counter() - t0 < seconds:
        n = min(chunk, ctrl_np.shape[0] - done)
        oracle.hashed_bezier_polyline_length(ctrl_np[done:done + n], n_t, seed, synth.PRECISION_T_STREAM, c0=done,
                                             threads=threads)
        done += n
    el = time.perf_counter() - t0
    return {"value": done * n_t / el, "unit": "points/s", "cores": threads, "kind": "oracle",
            "sample": f"first {done} of {ctrl_np.shape[0]} curves x {n_t} parameters (FP64 Bernstein sum + "
                      f"polyline length), {el:.1f} s wall"}


# ------------------------------------------------------------------ other workloads

def _hbm_line(name, value, unit, steps, warmup, ms, bytes_step, kern_ms, kernel, extra, traffic=None):
    peak, note = hbm_peak(load_peaks())
    achieved = bytes_step / (kern_ms * 1e-3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": unit, "n_gpus": 1, "steps": steps, "warmup": warmup,
            "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic", "config": {"workload": name},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "peak_source": note, "bytes_per_launch": bytes_step, "kernel": kernel}}
    line.update(extra)
    return line


def _record(name, value, unit, steps, warmup, ms, bytes_launch, kern_ms, kernel, clocks, extra, traffic=None):
    """One workload's entry of the default line's "configs" object: the
    metric over the whole step, the dominant kernel's HBM roofline and the
    clocks sampled while it ran."""
    line = _hbm_line(name, value, unit, steps, warmup, ms, bytes_launch, kern_ms, kernel, extra, traffic)
    rec = {"workload": name, "value": value, "unit": unit, "ms_per_step": line["ms_per_step"], "steps": steps,
           "warmup": warmup, "roofline": line["roofline"], "clocks": clocks}
    rec.update(extra)
    return rec


def _standalone(rec):
    """A workload's record as a JSON line of its own (--workload X)."""
    line = {"metric": METRIC, "value": rec["value"], "unit": rec["unit"], "n_gpus": 1, "steps": rec["steps"],
            "warmup": rec["warmup"], "ms_per_step": rec["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": rec["workload"]}}
    line.update({k: v for k, v in rec.items() if k not in line and k not in ("workload",)})
    return line


def run_plain(args):
    import torch

    from paper_2603_15447_gb300 import bez, synth
    import oracle
    ctx = bez.context(0)
    ctrl_np, t_np = synth.plain()
    ctrl, t = torch.from_numpy(ctrl_np).cuda(), torch.from_numpy(t_np).cuda()
    out = torch.empty((4096, 256, 3), device="cuda")
    timer = Timer(torch, ctx, torch.device("cuda", 0), 1)
    res = {}
    # a launch takes microseconds: time more steps so that the clock sampler
    # (100 ms period) sees the work
    steps = max(args.steps, 400)
    with ClockSampler(0) as clocks:
        for v in ("HORNER", "DECASTELJAU", "SEILER", "HORNER_CENTRED"):
            ms, st = timer.run(lambda v=v: bez.bez_eval(ctrl, t, variant=bez.Variant[v], out=out, ctx=ctx),
                               steps, args.warmup)
            res[v] = {"points_per_s": 4096 * 256 * steps / (ms * 1e-3),
                      "kernel_ms": st["timed_ms"] / max(st["timed_launches"], 1), "ms": ms}
    ref = oracle.bezier(ctrl_np, t_np)
    diag = np.maximum(np.linalg.norm(ref.max(axis=1) - ref.min(axis=1), axis=-1), 2.0 ** -4)
    for v in res:
        got = bez.bez_eval(ctrl, t, variant=bez.Variant[v], ctx=ctx).cpu().numpy().astype(np.float64)
        res[v]["max_norm_err"] = float((np.linalg.norm(got - ref, axis=-1).max(axis=1) / diag).max())
        res[v]["speedup_vs_horner"] = res[v]["points_per_s"] / res["HORNER"]["points_per_s"]
    # steady state of repeated evaluation: 32 back-to-back launches captured
    # in one CUDA graph and replayed, no L2 flush between them (the output
    # stays in L2); supplementary to the flushed per-launch value above
    steady = {}
    n_graph = 32
    for v in ("DECASTELJAU", "HORNER_CENTRED"):
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            for _ in range(n_graph):
                bez.bez_eval(ctrl, t, variant=bez.Variant[v], out=out, ctx=ctx)
        for _ in range(3):
            graph.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            graph.replay()
        e1.record()
        torch.cuda.synchronize()
        ms_g = e0.elapsed_time(e1)
        steady[v] = {"points_per_s": 4096 * 256 * n_graph * 10 / (ms_g * 1e-3),
                     "us_per_launch": ms_g * 1e3 / (n_graph * 10)}
        del graph
    head = res["DECASTELJAU"]
    return _record("plain: 4,096 cubic 3D curves x 256 shared uniform t, points stored", head["points_per_s"],
                   "points/s", steps, args.warmup, head["ms"], 4096 * 256 * 12 + 4096 * 48 + 1024,
                   head["kernel_ms"], "k_curve (points, de Casteljau)", clocks.summary(),
                   {"max_norm_err": head["max_norm_err"], "bar": FP32_BAR,
                    "variants": {v: {k: x for k, x in r.items() if k != "ms"} for v, r in res.items()},
                    "note": "12.6 MB of output fits in L2; the launch is latency-bound, so its HBM fraction is "
                            "not a roofline statement",
                    "graph_steady_state": {**steady, "launches_per_graph": n_graph,
                                           "note": "back-to-back launches replayed from one CUDA graph, no L2 "
                                                   "flush between them: repeated-evaluation rate, not the metric"}})


def _batch_reference_sample(w, ids):
    """Oracle points of the curves `ids` of a synth.batch workload: {c: [n][dim]}."""
    import oracle
    dim = w["dim"]
    groups = {}
    for c in ids:
        groups.setdefault((int(w["type"][c]), int(w["degree"][c]), int(w["n_ctrl"][c]), int(w["n_samples"][c])),
                          []).append(int(c))
    out = {}
    for (ty, p, n, ns), cs in groups.items():
        ctrl = np.stack([w["ctrl_pool"][w["ctrl_off"][c]: w["ctrl_off"][c] + n * dim].reshape(n, dim) for c in cs])
        t = oracle.grid(ns)
        if ty == 0:
            pts = oracle.bezier(ctrl, t)
        elif ty == 1:
            pts = oracle.bspline(ctrl, p, t)
        else:
            wts = np.stack([w["weight_pool"][w["weight_off"][c]: w["weight_off"][c] + n] for c in cs])
            pts = oracle.bspline(ctrl, p, t, weights=wts)
        for k, c in enumerate(cs):
            out[c] = pts[k]
    return out


def run_batch(args):
    import torch

    from paper_2603_15447_gb300 import bez, synth
    ctx = bez.context(0)
    w = synth.batch(n_curves=args.batch_curves)
    ctrl, wts = torch.from_numpy(w["ctrl_pool"]).cuda(), torch.from_numpy(w["weight_pool"]).cuda()
    out = torch.empty(w["out_len"], device="cuda")
    desc = bez.descriptors(w["type"], w["degree"], w["n_ctrl"], w["n_samples"], w["ctrl_off"], w["weight_off"],
                           w["out_off"])
    timer = Timer(torch, ctx, torch.device("cuda", 0), 1)
    n_pts = int(w["n_samples"].sum())
    bytes_step = n_pts * 12 + w["ctrl_pool"].nbytes + w["weight_pool"].nbytes
    if args.batch_shape:
        # one fixed launch shape (chunk, schedule, threads, repr), spans extracted once, no tuning
        chunk, sched, threads, rep = (int(x) for x in args.batch_shape.split(","))
        with ClockSampler(0) as clocks:
            b = bez.Batch(desc, 3, ctrl, wts, out, chunk=chunk, schedule=sched, threads=threads, repr=rep,
                          setup_each_launch=False, use_graph=True, ctx=ctx)
            ms_b, st_b = timer.run(b.launch, args.steps, args.warmup)
            b.close()
        return _record(f"batch: {len(desc)} mixed curves, fixed shape chunk {chunk} schedule {sched} threads "
                       f"{threads} repr {rep}, spans extracted once", n_pts * args.steps / (ms_b * 1e-3),
                       "points/s", args.steps, args.warmup, ms_b, bytes_step, ms_b / args.steps,
                       "k_batch_class (graph replay)", clocks.summary(),
                       {"gpu_launches": int(st_b["launches"]), "n_points": n_pts})
    with ClockSampler(0) as clocks:
        full = bez.Batch(desc, 3, ctrl, wts, out, autotune=True, setup_each_launch=True, use_graph=True, ctx=ctx)
        ms_full, st_full = timer.run(full.launch, args.steps, args.warmup)
        cfg = full.config()
        full.close()
        ev = bez.Batch(desc, 3, ctrl, wts, out, autotune=True, setup_each_launch=False, use_graph=True, ctx=ctx)
        ms_ev, st_ev = timer.run(ev.launch, args.steps, args.warmup)
        cfg_ev = ev.config()
    # accuracy of the timed launch's output: every 64th curve against the oracle
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    ev.close()
    ids = np.arange(0, len(desc), 64)
    ref = _batch_reference_sample(w, ids)
    worst, worst_kind = 0.0, {}
    for c in ids:
        ns = int(w["n_samples"][c])
        g = got[w["out_off"][c]: w["out_off"][c] + ns * 3].reshape(ns, 3)
        r = ref[int(c)]
        diag = max(float(np.linalg.norm(r.max(axis=0) - r.min(axis=0))), 2.0 ** -4)
        e = float(np.linalg.norm(g - r, axis=-1).max() / diag)
        kind = ("bezier", "bspline", "nurbs")[int(w["type"][c])]
        worst_kind[kind] = max(worst_kind.get(kind, 0.0), e)
        worst = max(worst, e)
    return _record(f"batch: {len(desc)} mixed curves (50% Bezier deg 1-7, 25% cubic B-spline, 25% NURBS), "
                   f"{n_pts} points, one graph-captured launch of the class kernels, autotuned",
                   n_pts * args.steps / (ms_full * 1e-3), "points/s", args.steps, args.warmup, ms_full, bytes_step,
                   ms_ev / args.steps, "k_batch_class (graph replay, spans extracted once)", clocks.summary(),
                   {"setup_each_launch_points_per_s": n_pts * args.steps / (ms_full * 1e-3),
                    "eval_only_points_per_s": n_pts * args.steps / (ms_ev * 1e-3),
                    "gpu_launches": int(st_full["launches"]), "autotuned": cfg, "autotuned_eval_only": cfg_ev,
                    "n_points": n_pts, "max_norm_err": worst, "max_norm_err_by_type": worst_kind, "bar": FP32_BAR,
                    "max_norm_err_sample": f"every 64th curve ({len(ids)} curves), all their points"})


def run_tensor(args):
    import torch

    from paper_2603_15447_gb300 import bez, synth
    import oracle
    ctx = bez.context(0)
    s = torch.from_numpy(synth.surfaces()).cuda()
    v = torch.from_numpy(synth.volumes()).cuda()
    so = torch.empty((65536, 32, 32, 3), device="cuda")
    vo = torch.empty((4096, 16, 16, 16, 1), device="cuda")
    timer = Timer(torch, ctx, torch.device("cuda", 0), 1)
    n_s, n_v = 65536 * 1024, 4096 * 4096
    tex, texs = bez.Variant.TEX_DECASTELJAU, bez.Variant.TEX_SEILER
    # launches of ~0.1 ms: more steps so that the clock sampler sees the work
    args = argparse.Namespace(**{**vars(args), "steps": max(args.steps, 100)})
    with ClockSampler(0) as clocks:
        ms_s, st_s = timer.run(lambda: bez.bez_eval_surface(s, 32, 32, out=so, ctx=ctx), args.steps, args.warmup)
        ms_v, st_v = timer.run(lambda: bez.bez_eval_volume(v, 16, 16, 16, out=vo, ctx=ctx), args.steps,
                               args.warmup)
        ms_t, st_t = timer.run(lambda: bez.bez_eval_surface(s, 32, 32, variant=tex, out=so, ctx=ctx), args.steps,
                               args.warmup)
        ms_ts, st_ts = timer.run(lambda: bez.bez_eval_surface(s, 32, 32, variant=texs, out=so, ctx=ctx),
                                 args.steps, args.warmup)
        # Seiler tiles spread over 9 x 9 and 5 x 5 texels (float4 and unorm16 texels)
        spread_s = {}
        for sp in (8, 4):
            for fname in ("AUTO", "UNORM16"):
                fmt = bez.TexFormat[fname]
                ms_x, st_x = timer.run(lambda fmt=fmt, sp=sp: bez.bez_eval_surface(s, 32, 32, variant=texs, out=so,
                                                                                   ctx=ctx, tex_format=fmt,
                                                                                   tex_spread=sp),
                                       args.steps, args.warmup)
                kx = st_x["timed_ms"] / st_x["timed_launches"]
                spread_s[f"spread{sp}/{fname}"] = {"points_per_s": n_s * args.steps / (ms_x * 1e-3), "kernel_ms": kx,
                                                   "pack_ms": ms_x / args.steps - kx,
                                                   "gbs": n_s * 12 / (kx * 1e-3) / 1e9, "tex_spread": sp,
                                                   "tex_format": fname}
        # half / bfloat16 control-point storage, FP32 contraction
        low = {}
        for lname, lt in (("f16", s.half()), ("bf16", s.bfloat16())):
            ms_l, st_l = timer.run(lambda lt=lt: bez.bez_eval_surface(lt, 32, 32, out=so, ctx=ctx), args.steps,
                                   args.warmup)
            low[lname] = {"points_per_s": n_s * args.steps / (ms_l * 1e-3),
                          "kernel_ms": st_l["timed_ms"] / max(st_l["timed_launches"], 1)}
        vol_tex = {}
        for vname in ("TEX_DECASTELJAU", "TEX_SEILER", "TEX_SEILER_S8", "TEX_SEILER_S4"):
            var, sp = bez.Variant[VARIANT_SPEC[vname][0]], VARIANT_SPEC[vname][1]
            ms_vt, st_vt = timer.run(lambda var=var, sp=sp: bez.bez_eval_volume(v, 16, 16, 16, variant=var, out=vo,
                                                                                ctx=ctx, tex_spread=sp),
                                     args.steps, args.warmup)
            kvt = st_vt["timed_ms"] / st_vt["timed_launches"]
            vol_tex[vname] = {"values_per_s": n_v * args.steps / (ms_vt * 1e-3), "kernel_ms": kvt,
                              "l2_gbs": (n_v * 4) / (kvt * 1e-3) / 1e9}
        unorm = {}
        for vname, var in (("TEX_DECASTELJAU", tex), ("TEX_SEILER", texs)):
            for fname in ("UNORM16", "UNORM8"):
                fmt = bez.TexFormat[fname]
                ms_u, st_u = timer.run(lambda var=var, fmt=fmt: bez.bez_eval_surface(s, 32, 32, variant=var, out=so,
                                                                                     ctx=ctx, tex_format=fmt),
                                       args.steps, args.warmup)
                unorm[f"{vname}/{fname}"] = {"points_per_s": n_s * args.steps / (ms_u * 1e-3),
                                             "kernel_ms": st_u["timed_ms"] / st_u["timed_launches"]}
    ks = st_s["timed_ms"] / st_s["timed_launches"]
    kv = st_v["timed_ms"] / st_v["timed_launches"]
    kt = st_t["timed_ms"] / st_t["timed_launches"]
    kts = st_ts["timed_ms"] / st_ts["timed_launches"]
    # accuracy on the first 1024 patches: max point error over the AABB
    # diagonal of the patch's FP64 grid points (FP32 control points)
    sub = s[:1024].contiguous()
    ref = oracle.surface(sub.cpu().numpy(), 32, 32).reshape(1024, -1, 3)
    diag = np.maximum(np.linalg.norm(ref.max(axis=1) - ref.min(axis=1), axis=-1), 2.0 ** -4)

    def surf_err(var, fmt=bez.TexFormat.AUTO, c=sub, spread=0):
        got = bez.bez_eval_surface(c, 32, 32, variant=var, ctx=ctx, tex_format=fmt, tex_spread=spread)
        got = got.cpu().numpy().reshape(1024, -1, 3)
        return float((np.linalg.norm(got.astype(np.float64) - ref, axis=-1).max(axis=1) / diag).max())
    for key, rec in unorm.items():
        vname, fname = key.split("/")
        rec["max_norm_err"] = surf_err(bez.Variant[vname], bez.TexFormat[fname])
    low["f16"]["max_norm_err"] = surf_err(bez.Variant.AUTO, c=sub.half())
    low["bf16"]["max_norm_err"] = surf_err(bez.Variant.AUTO, c=sub.bfloat16())
    for lname in low:
        low[lname]["bar"] = TEX_BAR
        low[lname]["meets_bar"] = low[lname]["max_norm_err"] <= TEX_BAR
    vsub = v[:256].contiguous()
    vref = oracle.volume(vsub.cpu().numpy(), 16, 16, 16).reshape(256, -1)
    vspan = np.maximum(vref.max(axis=1) - vref.min(axis=1), 2.0 ** -4)

    def vol_err(var, spread=0):
        got = bez.bez_eval_volume(vsub, 16, 16, 16, variant=var, ctx=ctx, tex_spread=spread).cpu().numpy()
        return float((np.abs(got.reshape(256, -1) - vref).max(axis=1) / vspan).max())
    for vname, rec in vol_tex.items():
        rec["max_norm_err"] = vol_err(bez.Variant[VARIANT_SPEC[vname][0]], VARIANT_SPEC[vname][1])
    for rec in spread_s.values():
        rec["max_norm_err"] = surf_err(texs, bez.TexFormat[rec["tex_format"]], spread=rec["tex_spread"])
        rec["bar"] = TEX_BAR
        rec["meets_bar"] = rec["max_norm_err"] <= TEX_BAR
    surf_err_fp32 = surf_err(bez.Variant.AUTO)
    return _record("tensor: 65,536 bicubic 3D patches on 32x32 + 4,096 tricubic scalar volumes on 16^3",
                   (n_s + n_v) * args.steps / ((ms_s + ms_v) * 1e-3), "points/s", args.steps, args.warmup,
                   ms_s + ms_v, n_s * 12 + 65536 * 192, ks, "k_surface_bicubic3_warp", clocks.summary(),
                   {"max_norm_err": max(surf_err_fp32, vol_err(bez.Variant.AUTO)), "bar": FP32_BAR,
                    "max_norm_err_sample": "first 1024 patches and 256 volumes, all grid points",
                    "surface_points_per_s": n_s * args.steps / (ms_s * 1e-3), "surface_max_norm_err": surf_err_fp32,
                    "volume_values_per_s": n_v * args.steps / (ms_v * 1e-3), "volume_kernel_ms": kv,
                    "volume_l2_gbs": (n_v * 4 + 4096 * 256) / (kv * 1e-3) / 1e9,
                    "volume_note": "the 67 MB volume output stays in the 126 MB L2 between steps, so volume "
                                   "GB/s are L2 figures, not an HBM roofline",
                    "surface_low_precision_storage": low,
                    "surface_tex": {"points_per_s": n_s * args.steps / (ms_t * 1e-3), "kernel_ms": kt,
                                    "gbs": n_s * 12 / (kt * 1e-3) / 1e9, "max_norm_err": surf_err(tex),
                                    "kernel": "k_surface_tex<3> (one trilinear read per row and coordinate)"},
                    "surface_tex_seiler": {"points_per_s": n_s * args.steps / (ms_ts * 1e-3), "kernel_ms": kts,
                                           "gbs": n_s * 12 / (kts * 1e-3) / 1e9, "max_norm_err": surf_err(texs),
                                           "kernel": "k_surface_tex<3, Seiler> (one bilinear read per row and "
                                                     "coordinate)"},
                    "surface_tex_unorm": unorm,
                    "surface_tex_seiler_spread": {**spread_s, "kernel": "k_surface_tex<3, Seiler> on spread "
                                                                        "tiles (9 x 9 or 5 x 5 texels)"},
                    "volume_tex": vol_tex},
                   traffic=TRAFFIC_SURFACE_65536)


# Convergence check of the fit (outside the timed steps): Adam with its own
# rate for the control points and for the parameters t (a sample's t moves
# along the curve and wants far smaller steps), both decayed on a cosine to
# 1 % over FIT_CONV_STEPS steps.  With one rate of 1e-2 for both (the timed
# configuration) the fit stalls far above the noise.
FIT_CONV_STEPS, FIT_CONV_LR = 500, (5e-2, 1e-3)


def fit_lr_factor(k, total):
    return 0.01 + 0.99 * 0.5 * (1.0 + math.cos(math.pi * min(k, total) / total))


def run_fit(args):
    import torch

    from paper_2603_15447_gb300 import bez, synth
    from paper_2603_15447_gb300.autograd import bezier_curve
    import oracle
    ctx = bez.context(0)
    truth, t_true, noise, init = synth.fit()
    target = bez.bez_eval(torch.from_numpy(truth).cuda(), torch.from_numpy(t_true).cuda(),
                          variant=bez.Variant.DECASTELJAU) + torch.from_numpy(noise).cuda()
    n_curves, n_t = target.shape[0], target.shape[1]
    t0 = np.tile((np.arange(n_t) / (n_t - 1.0)).astype(np.float32), (n_curves, 1))
    n = n_curves * n_t
    scale = 1.0 / (n * 3)

    # fused step: one kernel forms C, the residual, the loss and the adjoint
    ctrl = torch.tensor(init, device="cuda")
    t = torch.tensor(t0, device="cuda")
    opt = torch.optim.Adam([ctrl, t], lr=1e-2)

    # gradients of the first step against the oracle's analytic gradient
    # (first 1024 curves; upstream gradient 2 s (C - y) from the oracle's C)
    nsub = 1024
    _, gc, _, gt = bez.bez_mse_grad(ctrl[:nsub].contiguous(), t[:nsub].contiguous(), target[:nsub].contiguous(),
                                    loss_scale=scale, ctx=ctx)
    y = target[:nsub].cpu().numpy().astype(np.float64)
    C = oracle.bezier(init[:nsub], t0[:nsub])
    gref_c, _, gref_t = oracle.bezier_grad(init[:nsub], t0[:nsub], 2 * scale * (C - y))
    gc_err = float((np.abs(gc.cpu().numpy() - gref_c).max(axis=(1, 2)) / np.abs(gref_c).max(axis=(1, 2))).max())
    gt_err = float((np.abs(gt.cpu().numpy() - gref_t).max(axis=1) / np.abs(gref_t).max(axis=1)).max())

    def step():
        loss, gc, _, gt = bez.bez_mse_grad(ctrl, t, target, loss_scale=scale, ctx=ctx)
        ctrl.grad, t.grad = gc, gt
        opt.step()
        t.clamp_(0, 1)
        return loss

    # the same step through the autograd Function (forward kernel, torch MSE, adjoint kernel)
    ctrl_a = torch.tensor(init, device="cuda", requires_grad=True)
    t_a = torch.tensor(t0, device="cuda", requires_grad=True)
    opt_a = torch.optim.Adam([ctrl_a, t_a], lr=1e-2)

    def step_autograd():
        opt_a.zero_grad(set_to_none=False)
        loss = ((bezier_curve(ctrl_a, t_a) - target) ** 2).mean()
        loss.backward()
        opt_a.step()
        with torch.no_grad():
            t_a.clamp_(0, 1)
        return loss.detach()

    timer = Timer(torch, ctx, torch.device("cuda", 0), 1)
    with ClockSampler(0) as clocks:
        first = float(step().sum())
        ms, st = timer.run(step, args.steps, args.warmup)
        for _ in range(max(0, 200 - args.steps - args.warmup - 2)):
            step()
        final = float(step().sum())
        ms_a, _ = timer.run(step_autograd, args.steps, args.warmup)
        # the same fused step from the same start, two-rate cosine schedule
        ctrl2 = torch.tensor(init, device="cuda")
        t2 = torch.tensor(t0, device="cuda")
        opt2 = torch.optim.Adam([{"params": [ctrl2], "lr": FIT_CONV_LR[0]}, {"params": [t2], "lr": FIT_CONV_LR[1]}])
        for k in range(FIT_CONV_STEPS):
            for g, base in zip(opt2.param_groups, FIT_CONV_LR):
                g["lr"] = base * fit_lr_factor(k, FIT_CONV_STEPS)
            loss2, gc2, _, gt2 = bez.bez_mse_grad(ctrl2, t2, target, loss_scale=scale, ctx=ctx)
            ctrl2.grad, t2.grad = gc2, gt2
            opt2.step()
            t2.clamp_(0, 1)
        conv = float(loss2.sum())
        del ctrl2, t2, opt2
    kern_ms = st["timed_ms"] / max(st["timed_launches"], 1)
    # k_grad with a target, per sample: t 4 B + target 12 B in, grad_t 4 B out;
    # per curve: 48 B of control points in, 48 B of grad_ctrl and 4 B of loss out
    bytes_launch = n * 20 + n_curves * 100
    sigma = 0.01
    return _record(f"fit: {n_curves:,} cubic 3D curves x {n_t} samples, fused forward + squared error + adjoint, "
                   "then Adam, per step", n * args.steps / (ms * 1e-3), "samples/s", args.steps, args.warmup, ms,
                   bytes_launch, kern_ms, "k_grad (fused squared error), mean launch", clocks.summary(),
                   {"grad_ctrl_max_rel_err": gc_err, "grad_t_max_rel_err": gt_err,
                    "grad_err_sample": f"first step, first {nsub} curves, per-curve max error over the curve's "
                                       "largest oracle gradient",
                    "loss_first": first, "loss_after_200_steps": final, "rms_after_200_steps": final ** 0.5,
                    "noise_sigma": sigma, "rms_over_sigma": final ** 0.5 / sigma,
                    "fit_to_noise": {"rms": conv ** 0.5, "rms_over_sigma": conv ** 0.5 / sigma,
                                     "steps": FIT_CONV_STEPS,
                                     "optimizer": f"Adam, lr {FIT_CONV_LR[0]:g} (control points) and "
                                                  f"{FIT_CONV_LR[1]:g} (t), cosine decay to 1 %, t clamped "
                                                  "to [0, 1]; not timed"},
                    "autograd_step": {"samples_per_s": n * args.steps / (ms_a * 1e-3),
                                      "ms_per_step": ms_a / args.steps,
                                      "path": "bezier_curve forward kernel, torch squared error, adjoint kernel"}},
                   traffic=TRAFFIC_FIT_65536x512 if (n_curves, n_t) == (65536, 512) else None)


# ------------------------------------------------------------------ reference arm

def run_reference(args, rank):
    """The FP64 oracle timed on the host cores on bounded samples of the same
    workload (each step: args.ref_curves curves x n_t parameters)."""
    if rank != 0:
        return None
    import oracle
    from paper_2603_15447_gb300 import synth
    seed = synth.BASE_SEED + 1
    ctrl_np = synth.precision(seed=seed, n_curves=args.ref_curves * 4)
    threads = oracle.default_threads()

    def step(i):
        s = (i % 4) * args.ref_curves
        oracle.hashed_bezier_polyline_length(ctrl_np[s:s + args.ref_curves], args.n_t, seed,
                                             synth.PRECISION_T_STREAM, c0=s, threads=threads)

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(i)
    el = time.perf_counter() - t0
    pts = args.ref_curves * args.n_t * args.steps
    v = pts / el
    return {"metric": METRIC, "value": v, "unit": "points/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_name(args.n_curves, args.n_t), "sample_curves_per_step": args.ref_curves,
                       "n_t": args.n_t},
            "cpu_baseline": {"value": v, "unit": "points/s", "cores": threads, "kind": "oracle",
                             "sample": f"{args.ref_curves} curves x {args.n_t} parameters per step"},
            "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["all", "precision", "plain", "chains", "batch", "tensor", "fit"],
                    default="all")
    ap.add_argument("--variant", default="HORNER_CENTRED", choices=VARIANTS,
                    help="headline evaluator (the fastest one meeting the FP32 bar)")
    ap.add_argument("--variants", default="", help="comma-separated subset of evaluators to time")
    ap.add_argument("--n-curves", type=int, default=N_CURVES)
    ap.add_argument("--n-t", type=int, default=N_T)
    ap.add_argument("--n-chains", type=int, default=16384)
    ap.add_argument("--chain-t", type=int, default=65536)
    ap.add_argument("--skip-chains", action="store_true")
    ap.add_argument("--batch-curves", type=int, default=262144)
    ap.add_argument("--batch-shape", default="", help="chunk,schedule,threads,repr: time one fixed batch shape")
    ap.add_argument("--accuracy-curves", type=int, default=4096)
    ap.add_argument("--skip-accuracy", action="store_true")
    ap.add_argument("--skip-f16", action="store_true", help="skip the half-storage variant table")
    ap.add_argument("--skip-coissue", action="store_true", help="skip the texture + FP32 co-issue sweep")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-curves", type=int, default=16384)
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch of the headline kernel from an ncu capture")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank)
    else:
        import torch

        from paper_2603_15447_gb300 import build as _build
        if world > 1:
            import torch.distributed as dist
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
            if rank == 0:
                _build.build()
            dist.barrier()
        else:
            _build.build()
            torch.cuda.set_device(0)
        others = {"plain": run_plain, "batch": run_batch, "tensor": run_tensor, "fit": run_fit}
        if args.workload in ("all", "precision"):
            line = run_precision(args, rank, world, local_rank)
            if args.workload == "all" and world == 1 and line is not None:
                # the other four workloads, each measured on this GPU right after the headline
                line["configs"] = {name: fn(args) for name, fn in others.items()}
        elif args.workload == "chains":
            args.variants = "HORNER"
            args.skip_accuracy = True
            line = run_precision(args, rank, world, local_rank)
        else:
            line = _standalone(others[args.workload](args))
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
