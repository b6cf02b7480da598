"""The multi-GPU paths: N independent replicas of the single-mesh step (a
mesh does not shard), and the batched form's instances split into
contiguous ranges, one per rank, with no exchange.  The job's time is the
slowest rank's and its throughput counts every rank's units.  Checked with
world_size-2 gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench
from paper_2605_04773_gb300 import scenes


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=ws)
    try:
        got = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 0.5], ws, torch.device("cpu"))
        q.put((rank, got, bench.replica_throughput(ws, 100, got[0])))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_throughput_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, got, thr in out:
        assert got == [2.0, 10.0, 0.5]
        assert thr == pytest.approx(2 * 100 / 2.0)


def test_single_rank_is_the_identity():
    assert bench.max_over_ranks([3.0, 4.0], 1, None) == [3.0, 4.0]
    assert bench.replica_throughput(1, 10, 2.0) == 5.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = bench.argparse.Namespace(steps=1, warmup=0, impl="reference", gpus=2)
    bench.run_reference(args)   # returns at once, prints nothing
    assert capsys.readouterr().out == ""


def test_shard_instances_tile_and_balance():
    counts = scenes.instance_vertex_counts(n_inst=256)
    for ws in (1, 2, 3, 4, 8):
        ranges = [bench.shard_instances(counts, ws, k) for k in range(ws)]
        assert ranges[0][0] == 0 and ranges[-1][1] == counts.size
        assert all(ranges[k][1] == ranges[k + 1][0] for k in range(ws - 1))
        loads = [int(counts[a:b].sum()) for a, b in ranges]
        # each boundary is the first instance past k / ws of the vertices
        assert max(loads) - counts.sum() / ws <= counts.max()
    # a rank's sub-batch holds exactly the whole batch's instances
    sub = scenes.batch_instances(n_inst=3, first=5)
    full = scenes.batch_instances(n_inst=8)
    assert np.array_equal(np.diff(sub.vert_ptr), np.diff(full.vert_ptr)[5:8])
    assert np.array_equal(sub.dims, full.dims[5:8]) and np.array_equal(sub.frac, full.frac[5:8])


def _shard_worker(rank, ws, port, q):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=ws)
    try:
        counts = scenes.instance_vertex_counts(n_inst=256)
        a, b = bench.shard_instances(counts, ws, rank)
        mine = scenes.instance_vertex_counts(n_inst=b - a, first=a)
        # a per-rank "batch time" proportional to its vertices; the job's is the max
        t = float(mine.sum()) * 1e-6
        job = bench.max_over_ranks([t], ws, torch.device("cpu"))[0]
        q.put((rank, (a, b), int(mine.sum()), job, bench.replica_throughput(1, 256, job)))
    finally:
        dist.destroy_process_group()


def test_sharded_batch_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    counts = scenes.instance_vertex_counts(n_inst=256)
    (r0, ra, va, ja, tha), (r1, rb, vb, jb, thb) = out
    assert ra[0] == 0 and ra[1] == rb[0] and rb[1] == 256
    assert va + vb == int(counts.sum())
    assert ja == jb == max(va, vb) * 1e-6
    assert tha == thb == pytest.approx(256 / ja)
