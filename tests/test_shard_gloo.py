"""The multi-rank path on CPU: two gloo processes each take their balanced
shard of a mixed batch, evaluate it (with the oracle, since this runs without
a GPU) and the gathered results equal a single-process evaluation.  The only
collective here is the test's own gather; evaluation exchanges nothing."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _evaluate(w, lo, hi):
    import oracle
    dim = w["dim"]
    out = []
    for c in range(lo, hi):
        n, p, ns, ty = int(w["n_ctrl"][c]), int(w["degree"][c]), int(w["n_samples"][c]), int(w["type"][c])
        ctrl = w["ctrl_pool"][w["ctrl_off"][c]: w["ctrl_off"][c] + n * dim].reshape(1, n, dim)
        t = oracle.grid(ns)
        if ty == 0:
            pts = oracle.bezier(ctrl, t, threads=1)
        else:
            wts = None if ty == 1 else w["weight_pool"][w["weight_off"][c]: w["weight_off"][c] + n].reshape(1, n)
            pts = oracle.bspline(ctrl, p, t, weights=wts, threads=1)
        out.append(pts.ravel())
    return np.concatenate(out) if out else np.zeros(0)


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import torch
    import torch.distributed as dist

    from paper_2603_15447_gb300 import shard, synth
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    w = synth.batch(n_curves=200, max_samples=64)
    lo, hi = shard.shard_of(w["n_samples"], rank, world)
    mine = torch.from_numpy(_evaluate(w, lo, hi))
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([mine.numel()]))
    # shards differ in size: pad to the largest, gather, trim
    m = max(int(s) for s in sizes)
    padded = torch.zeros(m, dtype=torch.float64)
    padded[: mine.numel()] = mine
    gathered = [torch.zeros(m, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, padded)
    parts = [g[: int(s)] for g, s in zip(gathered, sizes)]
    if rank == 0:
        q.put((np.concatenate([p.numpy() for p in parts]), [int(s) for s in sizes]))
    dist.destroy_process_group()


def test_balanced_ranges_partition_and_balance():
    from paper_2603_15447_gb300 import shard, synth
    w = synth.batch(n_curves=5000)
    for world in (1, 2, 3, 8):
        rs = shard.balanced_ranges(w["n_samples"], world)
        assert rs[0][0] == 0 and rs[-1][1] == 5000
        assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
        work = [int(w["n_samples"][a:b].sum()) for a, b in rs]
        assert max(work) - min(work) <= 2 * int(w["n_samples"].max())


def test_two_gloo_ranks_match_single_process():
    mp = pytest.importorskip("torch.multiprocessing")
    from paper_2603_15447_gb300 import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, sizes = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    w = synth.batch(n_curves=200, max_samples=64)
    want = _evaluate(w, 0, 200)
    assert len(sizes) == 2 and sum(sizes) == want.size
    np.testing.assert_array_equal(got, want)
