"""The benchmark's output contract, checked on the CPU through the reference
arm (the FP64 oracle timed on the host cores): one JSON line with the keys
and types a consumer of bench.py relies on, for a tiny sample of the
default workload."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run_reference():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--ref-curves", "32", "--n-t", "64"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_line_keys_and_types():
    d = _run_reference()
    for k, typ in (("metric", str), ("value", float), ("unit", str), ("n_gpus", int), ("steps", int),
                   ("warmup", int), ("ms_per_step", float), ("higher_is_better", bool), ("scaling", str),
                   ("dtype", str), ("data", str), ("config", dict), ("impl", str), ("cpu_baseline", dict),
                   ("e2e", dict)):
        assert isinstance(d[k], typ), (k, d.get(k))
    assert d["impl"] == "reference" and d["vs_baseline"] is None
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["scaling"] == "weak" and d["data"] == "synthetic" and d["value"] > 0
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert isinstance(cb["sample"], str) and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_roofline_block_arithmetic():
    # the roofline object of a bandwidth-bound line: achieved = algorithmic
    # bytes per launch / launch time, frac = achieved / peak, peak from the
    # measured copy bandwidth or the stated fallback
    sys.path.insert(0, ROOT)
    import bench
    line = bench._hbm_line("w", 1.0, "points/s", 3, 3, 6.0, 10 ** 9, 0.5, "k", {"extra": 1}, traffic=123.0)
    r = line["roofline"]
    assert set(("bound", "achieved", "peak", "unit", "frac", "traffic")) <= set(r)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] == 123.0
    assert abs(r["achieved"] - 2000.0) < 1e-9                    # 1e9 B in 0.5 ms
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    peak, note = bench.hbm_peak(bench.load_peaks())
    assert r["peak"] == peak and ("measured" in note or "fallback" in note)
    assert bench.hbm_peak(None) == (6800.0, "of fallback (6.8 TB/s)")
    assert line["extra"] == 1 and line["ms_per_step"] == 2.0 and line["config"] == {"workload": "w"}
    ops, note = bench.alu_peak(None)
    assert ops == 152 * 128 * 2070.0e6 and "fallback" in note
    ops, note = bench.alu_peak({"sm_max_mhz": 2000.0}, sms=100)
    assert ops == 100 * 128 * 2000.0e6 and "device" in note


def test_variant_table_and_fit_schedule():
    # the spread texture variants resolve to TEX_SEILER with their spread,
    # every texture variant has a fetch count and an eval op count, and the
    # fit convergence check's cosine schedule starts at the full rate, ends
    # at 1 % and never rises
    import bench
    assert bench.VARIANT_SPEC["TEX_SEILER_S8"] == ("TEX_SEILER", 8)
    assert bench.VARIANT_SPEC["TEX_SEILER_S4"] == ("TEX_SEILER", 4)
    for v in bench.TEX_VARIANTS:
        assert v in bench.TEX_FETCHES and v in bench.EVAL_OPS
    assert set(bench.VARIANT_SPEC) == set(bench.VARIANTS)
    T = bench.FIT_CONV_STEPS
    f = [bench.fit_lr_factor(k, T) for k in range(T + 1)]
    assert f[0] == 1.0 and abs(f[-1] - 0.01) < 1e-12
    assert all(a >= b for a, b in zip(f, f[1:]))
    assert bench.fit_lr_factor(2 * T, T) == f[-1]
