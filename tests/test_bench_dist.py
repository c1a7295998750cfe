"""The multi-rank host logic of bench.py on CPU with gloo (world size 2):
every rank convexifies its own mesh (weak scaling), the timed region is the
slowest rank's, and the whole-job rate counts all ranks' points; the
reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

from conftest import ROOT


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    w, r, _ = bench.dist_env()
    t = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    F, _ = bench.make_inputs(4, rank)
    dist.barrier()
    q.put((r, w, t, float((F * F).sum()), F.shape[0], bench.whole_job_rate(F.shape[0], w, 3, t)))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_distinct_meshes():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, t0, s0, n0, v0), (r1, w1, t1, s1, n1, v1) = res
    assert (r0, r1) == (0, 1) and w0 == w1 == 2
    assert t0 == t1 == 15.0
    assert n0 == n1 == 64 and s0 != s1  # one mesh per rank, seeded by rank
    assert v0 == v1 == pytest.approx(2 * 64 * 3 / 0.015)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        nx, cpu_points, warmup, steps, gpus = 4, 1, 0, 1, 2

    assert bench.run_reference(A()) is None
    assert capsys.readouterr().out == ""


def _range_worker(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import numpy as np
    import torch
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    # expected tree size per point: 1 + 3 where the point is past its history
    w = 1.0 + 3.0 * (np.random.default_rng(5).random(10001) < 0.3)
    lo, hi = bench.rank_ranges(w, ws)[rank]
    t = torch.tensor([lo, hi], dtype=torch.int64)
    allr = [torch.zeros(2, dtype=torch.int64) for _ in range(ws)]
    dist.all_gather(allr, t)
    q.put((rank, [tuple(x.tolist()) for x in allr], float(w[lo:hi].sum()), float(w.sum())))
    dist.destroy_process_group()


def test_two_ranks_split_one_problem_into_weighted_contiguous_ranges():
    """Strong-scaling split: every rank computes the same contiguous ranges
    of one problem; together they cover it exactly once, and the expected
    tree sizes are balanced to within one point's weight."""
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_range_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, r0, w0, tot), (_, r1, w1, _) = res
    assert r0 == r1  # every rank derives the same split
    (a0, b0), (a1, b1) = r0
    assert a0 == 0 and b0 == a1 and b1 == 10001
    assert abs(w0 - w1) <= 4.0 and w0 + w1 == tot


def test_rank_ranges_edge_cases():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.rank_ranges([1.0] * 8, 4) == [(0, 2), (2, 4), (4, 6), (6, 8)]
    assert bench.rank_ranges([], 2) == [(0, 0), (0, 0)]
    r = bench.rank_ranges([5.0, 1, 1, 1, 1, 1], 2)
    assert r[0][0] == 0 and r[-1][1] == 6 and r[0][1] == r[1][0]
