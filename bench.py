"""Benchmark: curve points evaluated per second on the fused
evaluate-and-measure workload, per evaluator, against FP32 Horner on the same
GPU, with the max normalised error against the FP64 oracle.

Workload (one step): 1,048,576 cubic 3D Bezier curves (control points
U[-1,1]^3, FP32), each at 1024 parameters drawn U[0,1) inside the kernel,
evaluated and reduced to one polyline length per curve; no points are
stored.  A step is one bez_eval call: per-curve setup, parameter draw,
evaluation and the warp-shuffle length reduction, all in one kernel.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  Under torchrun (N > 1) every rank evaluates its own
batch of the same size (weak scaling, different seeds); the only
cross-rank traffic is the timing barrier and a max over ranks of the timed
duration.
"""
from __future__ import annotations

import argparse
import json
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
DEGREE = 3
DIM = 3
WORKLOAD = ("precision/texture: 1,048,576 cubic 3D Bezier curves (U[-1,1]^3 FP32), 1024 parameters per curve "
            "drawn U[0,1) in-kernel, fused per-curve polyline length (no point stores)")

# Algorithmic lane operations per point (cubic, 3D), see the design doc:
# parameter draw 12 (xor, lowbias32 = 3 shift + 3 xor + 2 mul, shift-or,
# subtract) + evaluation + polyline step 8 (3 sub, mul + 2 fma, sqrt, add).
T_OPS, LEN_OPS = 12, 8
EVAL_OPS = {"HORNER": 9, "HORNER_CENTRED": 10, "BERNSTEIN": 19, "SEILER": 16, "DECASTELJAU": 36}
VARIANTS = ["HORNER", "HORNER_CENTRED", "BERNSTEIN", "SEILER", "DECASTELJAU"]
FP32_BAR = 1e-6


def alu_peak(peaks):
    """FP32/INT32 lane-operation issue peak: 152 SMs x 128 lanes x max clock."""
    sms, lanes = 152, 128
    mhz = float(peaks.get("sm_max_mhz", 2070.0)) if peaks else 2070.0
    return sms * lanes * mhz * 1e6, f"152 SMs x 128 lanes x {mhz:.0f} MHz (derived from unit counts and max clock)"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return None


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


# ------------------------------------------------------------------ ours

def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2603_15447_gb300 import bez, synth
    from paper_2603_15447_gb300 import build as _build

    if rank == 0 or world == 1:
        _build.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    seed = synth.BASE_SEED + 1 + 1000 * rank
    ctrl_np = synth.precision(seed=seed, n_curves=args.n_curves)
    ctrl = torch.from_numpy(ctrl_np).to(dev)
    out = torch.empty(args.n_curves, dtype=torch.float32, device=dev)
    ctx = bez.context(local_rank)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # 256 MiB > 129 MB L2

    def step(variant):
        bez.bez_eval(ctrl, None, n_t=args.n_t, variant=bez.Variant[variant], out_mode=bez.OutMode.POLYLINE_LENGTH,
                     t_mode=bez.TMode.HASH, seed=seed, stream_id=synth.PRECISION_T_STREAM, out=out, ctx=ctx)

    def timed(variant, steps, warmup, sampler=None):
        for _ in range(warmup):
            step(variant)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ctx.reset_stats()
        ctx.set_timing(True)
        evs = []
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(variant)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_wall
        if world > 1:
            dist.barrier()
        ctx.set_timing(False)
        st = ctx.stats()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        return ms, st, wall

    results = {}
    headline = args.variant
    run_variants = [v for v in VARIANTS if v in args.variants.split(",")] if args.variants else list(VARIANTS)
    if headline not in run_variants:
        run_variants.append(headline)
    with ClockSampler(local_rank) as clocks:
        for v in run_variants:
            ms, st, wall = timed(v, args.steps, args.warmup)
            results[v] = {"ms": ms, "stats": st}
    clock_summary = clocks.summary()

    # max over ranks of the device time of the headline variant
    ms_head = results[headline]["ms"]
    if world > 1:
        t = torch.tensor([ms_head], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_head = float(t.item())

    # end to end through the public API with pinned host buffers
    ctrl_host = torch.from_numpy(ctrl_np).pin_memory()
    out_host = torch.empty(args.n_curves, dtype=torch.float32).pin_memory()

    def e2e_step():
        bez.bez_eval(ctrl_host, None, n_t=args.n_t, variant=bez.Variant[headline],
                     out_mode=bez.OutMode.POLYLINE_LENGTH, t_mode=bez.TMode.HASH, seed=seed,
                     stream_id=synth.PRECISION_T_STREAM, out=out_host, ctx=ctx)

    for _ in range(max(args.warmup, 1)):
        e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e2e_s = (time.perf_counter() - t0) / args.steps

    if rank != 0:
        return None

    pts_per_step = args.n_curves * args.n_t
    peaks = load_peaks()
    peak, peak_note = alu_peak(peaks)
    variants = {}
    for v in run_variants:
        r = results[v]
        st = r["stats"]
        kern_ms = st["timed_ms"] / max(st["timed_launches"], 1)
        ops = (T_OPS + EVAL_OPS[v] + LEN_OPS) * pts_per_step
        variants[v] = {"points_per_s": pts_per_step * args.steps / (r["ms"] * 1e-3),
                       "ms_per_step": r["ms"] / args.steps, "kernel_ms": kern_ms,
                       "alu_frac": ops / (kern_ms * 1e-3) / peak, "ops_per_point": T_OPS + EVAL_OPS[v] + LEN_OPS}
    horner = variants["HORNER"]["points_per_s"] if "HORNER" in variants else None
    for v in run_variants:
        variants[v]["speedup_vs_horner"] = variants[v]["points_per_s"] / horner if horner else None

    # accuracy on a sample of the same workload (points mode, same parameters)
    if not args.skip_accuracy:
        import oracle
        ns = args.accuracy_curves
        sample = ctrl[:ns].contiguous()
        th = oracle.hash_t(seed, synth.PRECISION_T_STREAM, 0, ns, args.n_t)
        ref = oracle.bezier(ctrl_np[:ns], th)
        diag = np.maximum(np.linalg.norm(ref.max(axis=1) - ref.min(axis=1), axis=-1), 2.0 ** -4)
        for v in run_variants:
            pts = bez.bez_eval(sample, None, n_t=args.n_t, variant=bez.Variant[v], t_mode=bez.TMode.HASH,
                               seed=seed, stream_id=synth.PRECISION_T_STREAM, ctx=ctx)
            err = np.linalg.norm(pts.cpu().numpy().astype(np.float64) - ref, axis=-1).max(axis=1) / diag
            variants[v]["max_norm_err"] = float(err.max())
            variants[v]["meets_1e-6"] = bool(err.max() <= FP32_BAR)

    head = variants[headline]
    kern_ms = head["kernel_ms"]
    ops_launch = head["ops_per_point"] * pts_per_step
    achieved = ops_launch / (kern_ms * 1e-3)
    line = {
        "metric": METRIC,
        "value": pts_per_step * world * args.steps / (ms_head * 1e-3),
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
        "config": {"workload": WORKLOAD, "variant": headline, "n_curves": args.n_curves, "n_t": args.n_t,
                   "degree": DEGREE, "dim": DIM, "l2": "flushed between timed steps (256 MiB device write)",
                   "speedup_vs_horner": head["speedup_vs_horner"]},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "Tops/s",
                     "frac": achieved / peak, "traffic": args.traffic, "peak_source": peak_note,
                     "ops_per_launch": ops_launch, "kernel": "k_curve (fused hash + eval + polyline length)"},
        "e2e": {"value": pts_per_step / e2e_s, "unit": "points/s",
                "h2d_bytes_per_step": int(ctrl_np.nbytes), "d2h_bytes_per_step": int(args.n_curves * 4)},
        "gpu_launches": int(results[headline]["stats"]["launches"]),
        "clocks": clock_summary,
        "variants": variants,
    }
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
            "config": {"workload": WORKLOAD, "sample_curves_per_step": args.ref_curves, "n_t": args.n_t},
            "cpu_baseline": {"value": v, "unit": "points/s", "cores": threads, "kind": "oracle",
                             "sample": f"{args.ref_curves} curves x {args.n_t} parameters per step"},
            "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--variant", default="HORNER_CENTRED", choices=VARIANTS)
    ap.add_argument("--variants", default="", help="comma-separated subset of evaluators to time")
    ap.add_argument("--n-curves", type=int, default=N_CURVES)
    ap.add_argument("--n-t", type=int, default=N_T)
    ap.add_argument("--accuracy-curves", type=int, default=4096)
    ap.add_argument("--skip-accuracy", action="store_true")
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
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
        line = run_ours(args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
