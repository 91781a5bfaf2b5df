"""Host logic of bench.py's multi-process path on CPU: world_size-2 gloo ranks
agree on the max-over-ranks time and the whole-job throughput; the
reference arm does its work on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank           # rank 1 is the slow one
    m = bench.max_over_ranks(ms)
    out[rank] = (m, bench.job_throughput(world, 10, m))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1]
    m, v = out[0]
    assert m == 150.0
    assert v == pytest.approx(2 * 10 / 0.150)


def test_reference_arm_skips_non_zero_ranks(monkeypatch, capsys):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    called = []
    monkeypatch.setattr(bench, "make_system", lambda: called.append(1))
    bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert called == [] and capsys.readouterr().out == ""


def test_single_rank_max_is_identity():
    import bench

    assert bench.max_over_ranks(12.5) == 12.5
