"""The multi-GPU path is N independent replicas (a single mesh does not
shard): the job's time is the slowest rank's and its throughput counts every
rank's units.  Checked with world_size-2 gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


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
