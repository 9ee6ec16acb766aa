"""GPU parity of mixed batches (bez_batch_*, bez_eval_batch): Bezier curves,
clamped uniform B-splines and NURBS of degrees 1..7 with log-uniform sample
counts, evaluated in one persistent launch (graph-captured, autotuned) and
compared curve by curve with the oracle at the FP32 bar."""
import numpy as np
import pytest

import oracle
from gpu_util import need_gpu, normalised_error

pytestmark = pytest.mark.gpu
FP32_BAR = 1e-6


def _reference(w):
    """Oracle points of every curve of a synth.batch workload, as one flat
    array laid out like out_pool."""
    dim = w["dim"]
    out = np.zeros(w["out_len"], np.float64)
    groups = {}
    for c in range(len(w["type"])):
        groups.setdefault((int(w["type"][c]), int(w["degree"][c]), int(w["n_ctrl"][c]), int(w["n_samples"][c])),
                          []).append(c)
    for (ty, p, n, ns), ids in groups.items():
        if ns == 0:
            continue
        ids = np.array(ids)
        ctrl = np.stack([w["ctrl_pool"][w["ctrl_off"][c]: w["ctrl_off"][c] + n * dim].reshape(n, dim) for c in ids])
        t = oracle.grid(ns)
        if ty == 0:
            pts = oracle.bezier(ctrl, t)
        elif ty == 1:
            pts = oracle.bspline(ctrl, p, t)
        else:
            wts = np.stack([w["weight_pool"][w["weight_off"][c]: w["weight_off"][c] + n] for c in ids])
            pts = oracle.bspline(ctrl, p, t, weights=wts)
        for k, c in enumerate(ids):
            out[w["out_off"][c]: w["out_off"][c] + ns * dim] = pts[k].ravel()
    return out


def _check_all(got, ref, w):
    dim = w["dim"]
    worst = 0.0
    for c in range(len(w["type"])):
        ns = int(w["n_samples"][c])
        if ns == 0:
            continue
        g = got[w["out_off"][c]: w["out_off"][c] + ns * dim].reshape(1, ns, dim)
        r = ref[w["out_off"][c]: w["out_off"][c] + ns * dim].reshape(1, ns, dim)
        worst = max(worst, float(normalised_error(g, r)[0]))
    return worst


@pytest.fixture(scope="module")
def workload():
    from paper_2603_15447_gb300 import synth
    w = synth.batch(n_curves=3000, max_samples=600)
    return w, _reference(w)


def _pools(torch, w):
    ctrl = torch.from_numpy(w["ctrl_pool"]).cuda()
    wts = torch.from_numpy(w["weight_pool"]).cuda()
    out = torch.full((w["out_len"],), float("nan"), device="cuda")
    return ctrl, wts, out


def _desc(w):
    from paper_2603_15447_gb300 import bez
    return bez.descriptors(w["type"], w["degree"], w["n_ctrl"], w["n_samples"], w["ctrl_off"], w["weight_off"],
                           w["out_off"])


@pytest.mark.parametrize("schedule,chunk,threads,repr", [(0, 256, 256, 1), (1, 512, 128, 0), (0, 2048, 128, 1),
                                                          (1, 1024, 256, 1), (0, 512, 256, 0), (2, 512, 128, 1),
                                                          (2, 256, 256, 0)])
def test_batch_plan_graph_replay(workload, schedule, chunk, threads, repr):
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    w, ref = workload
    ctrl, wts, out = _pools(torch, w)
    b = bez.Batch(_desc(w), w["dim"], ctrl, wts, out, chunk=chunk, schedule=schedule, threads=threads, repr=repr)
    for _ in range(2):
        out.fill_(float("nan"))
        b.launch()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert _check_all(got, ref, w) <= FP32_BAR
    assert b.config() == {"chunk": chunk, "schedule": schedule, "threads": threads, "repr": repr}
    b.close()


@pytest.mark.parametrize("dim", [1, 2, 4])
def test_batch_other_dims(dim):
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez, synth
    w = synth.batch(n_curves=400, max_samples=300, dim=dim)
    ref = _reference(w)
    ctrl, wts, out = _pools(torch, w)
    for repr in (0, 1):
        out.fill_(float("nan"))
        bez.Batch(_desc(w), dim, ctrl, wts, out, repr=repr).launch()
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        # scalar and 2D curves: normalise by the control polygon (secondary normaliser)
        for c in range(len(w["type"])):
            ns = int(w["n_samples"][c])
            if ns == 0:
                continue
            g = got[w["out_off"][c]: w["out_off"][c] + ns * dim].reshape(ns, dim)
            r = ref[w["out_off"][c]: w["out_off"][c] + ns * dim].reshape(ns, dim)
            cp = w["ctrl_pool"][w["ctrl_off"][c]: w["ctrl_off"][c] + int(w["n_ctrl"][c]) * dim].reshape(-1, dim)
            scale = max(np.linalg.norm(cp.max(axis=0) - cp.min(axis=0)), 2.0 ** -4)
            assert np.linalg.norm(g - r, axis=-1).max() / scale <= FP32_BAR


def test_batch_autotune_and_static_spans(workload, tmp_path, monkeypatch):
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    w, ref = workload
    monkeypatch.setenv("BEZ_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    ctrl, wts, out = _pools(torch, w)
    b = bez.Batch(_desc(w), w["dim"], ctrl, wts, out, autotune=True, setup_each_launch=False)
    cfg = b.config()
    assert cfg["chunk"] in (256, 512, 1024, 2048) and cfg["schedule"] in (0, 1, 2) and cfg["threads"] in (128, 256)
    out.fill_(float("nan"))
    b.launch()
    torch.cuda.synchronize()
    assert _check_all(out.cpu().numpy(), ref, w) <= FP32_BAR
    b.close()
    text = (tmp_path / "tune.json").read_text()
    assert '"chunk"' in text and "batch-v3:setup0" in text and '"partition"' in text
    # a second plan of the same shape and setup mode takes the cached choice
    b2 = bez.Batch(_desc(w), w["dim"], ctrl, wts, out, autotune=True, setup_each_launch=False)
    assert b2.config() == cfg
    b2.close()


def test_one_shot_and_empty_curves(workload):
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    w, ref = workload
    ctrl, wts, out = _pools(torch, w)
    bez.bez_eval_batch(_desc(w), w["dim"], ctrl, wts, out)
    assert _check_all(out.cpu().numpy(), ref, w) <= FP32_BAR
    d = _desc(w)[:10].copy()
    d["n_samples"][3] = 0
    d["n_samples"][4] = 1
    bez.bez_eval_batch(d, w["dim"], ctrl, wts, out)


def test_batch_rejects_bad_descriptors(workload):
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    w, _ = workload
    ctrl, wts, out = _pools(torch, w)
    for field, value in (("degree", 9), ("ctrl_off", 10 ** 12), ("out_off", -1), ("type", 5)):
        d = _desc(w)[:5].copy()
        d[field][2] = value
        with pytest.raises(bez.BezError) as e:
            bez.bez_eval_batch(d, w["dim"], ctrl, wts, out)
        assert e.value.status == bez.Status.INVALID_ARG and "curve 2" in str(e.value)
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval_batch(_desc(w)[:5], w["dim"], ctrl.cpu(), wts, out)
    assert e.value.status == bez.Status.INVALID_ARG


@pytest.mark.parametrize("repr", [0, 1])
def test_batch_grid_values_are_exact_quotients(repr):
    # Degree-1 Bezier curves from (0, 0, 0) to (1, 1, 1): with Bezier-point
    # spans (de Casteljau) every coordinate is lerp(0, 1, t) = t exactly, so
    # the output is the sample grid t_j = fl32(j) / fl32(n - 1) bit for bit
    # (the kernels form it without a division for n - 1 < 2^16, by division
    # above).  The centred power basis gives 1/2 + (t - 1/2): compared at 1e-7.
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    ns = np.array([1, 2, 3, 7, 255, 256, 1000, 4097, 65536, 65537, 70001], np.int32)
    n = len(ns)
    ctrl = np.tile(np.array([0, 0, 0, 1, 1, 1], np.float32), n)
    out_off = np.concatenate([[0], np.cumsum(ns.astype(np.int64) * 3)])
    d = bez.descriptors(np.zeros(n, np.int32), np.ones(n, np.int32), np.full(n, 2, np.int32), ns,
                        np.arange(n, dtype=np.int64) * 6, np.zeros(n, np.int64), out_off[:-1])
    out = torch.zeros(int(out_off[-1]), device="cuda")
    b = bez.Batch(d, 3, torch.from_numpy(ctrl).cuda(), torch.zeros(1, device="cuda"), out, repr=repr)
    b.launch()
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for c in range(n):
        m = int(ns[c])
        t = oracle.grid(m).astype(np.float32)
        pts = got[out_off[c]: out_off[c + 1]].reshape(m, 3)
        if repr == 0:
            for k in range(3):
                np.testing.assert_array_equal(pts[:, k], t)
        else:
            assert np.abs(pts - t[:, None]).max() <= 1e-7


def test_batch_full_sample_range_and_long_nurbs():
    # the batch workload's full range of sample counts (16..4096, log-uniform)
    # and degree-7 NURBS with 64 control points and long runs of samples per
    # curve (several work items each, many spans per item), every curve
    # against the oracle, under the tuned shape and the partitioned schedule
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez, synth
    w = synth.batch(n_curves=1500, max_samples=4096, seed=synth.BASE_SEED + 77)
    # a block of long degree-7 NURBS: 64 control points, 4096 and 3000 samples
    rng = np.random.default_rng(77)
    extra = 24
    base_c, base_w, base_o = len(w["ctrl_pool"]), len(w["weight_pool"]), w["out_len"]
    ns_extra = np.where(np.arange(extra) % 2 == 0, 4096, 3000).astype(np.int32)
    ctrl_x = rng.uniform(-1, 1, extra * 64 * 3).astype(np.float32)
    w_x = rng.uniform(0.5, 2, extra * 64).astype(np.float32)
    w = dict(w)
    w["type"] = np.concatenate([w["type"], np.full(extra, 2, np.int32)])
    w["degree"] = np.concatenate([w["degree"], np.full(extra, 7, np.int32)])
    w["n_ctrl"] = np.concatenate([w["n_ctrl"], np.full(extra, 64, np.int32)])
    w["n_samples"] = np.concatenate([w["n_samples"], ns_extra])
    w["ctrl_off"] = np.concatenate([w["ctrl_off"], base_c + np.arange(extra, dtype=np.int64) * 192])
    w["weight_off"] = np.concatenate([w["weight_off"], base_w + np.arange(extra, dtype=np.int64) * 64])
    w["out_off"] = np.concatenate([w["out_off"], base_o + np.concatenate([[0], np.cumsum(ns_extra[:-1] * 3)])])
    w["ctrl_pool"] = np.concatenate([w["ctrl_pool"], ctrl_x])
    w["weight_pool"] = np.concatenate([w["weight_pool"], w_x])
    w["out_len"] = int(base_o + ns_extra.sum() * 3)
    assert w["n_samples"].max() >= 4000 and w["n_samples"].min() <= 20
    ref = _reference(w)
    ctrl, wts, out = _pools(torch, w)
    for kw in (dict(autotune=True), dict(schedule=2, chunk=512, threads=128, repr=1),
               dict(schedule=2, chunk=1024, threads=256, repr=0)):
        b = bez.Batch(_desc(w), 3, ctrl, wts, out, **kw)
        out.fill_(float("nan"))
        b.launch()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert _check_all(got, ref, w) <= FP32_BAR, kw
        b.close()
