"""The multi-GPU form of the benchmark is replicas only: every rank decomposes its own
tensor, ranks meet at barriers, the job's time is the slowest rank's, and the reference
arm runs on rank 0 alone. Checked with two gloo ranks on the CPU."""

import multiprocessing as mp
import os
import socket

import pytest

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo")
    w, r, local = bench.dist_env()
    bench.barrier(w)
    # rank r spent 1 + r seconds on its 10 units of work
    value = bench.weak_scaling_value(10, 1.0 + r, w)
    bench.barrier(w)
    q.put((r, w, local, value))
    dist.destroy_process_group()


def test_replica_throughput_uses_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [(r, w, l) for r, w, l, _ in out] == [(0, 2, 0), (1, 2, 1)]
    # 2 ranks x 10 units over the slowest rank's 2 s, the same on every rank
    assert all(v == pytest.approx(10.0) for *_, v in out)


def test_single_process_value_is_local():
    assert bench.weak_scaling_value(10, 4.0, 1) == pytest.approx(2.5)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = bench.argparse.Namespace(gpus=2, steps=1, warmup=0)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
