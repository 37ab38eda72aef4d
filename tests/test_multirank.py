"""The N-GPU path of the benchmark (replicas: one process per GPU, no
data-path collective) on CPU with world size 2 over gloo.

* each rank's timed region is reduced to the slowest rank's (the job ends
  with its last replica), and whole-job throughput counts every replica's
  units over that time;
* the reference arm under a multi-rank launch prints from rank 0 only;
* the rank environment is read from RANK / WORLD_SIZE / LOCAL_RANK.
"""
import io
import os
import socket
import contextlib

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = 10.0 + 5.0 * rank  # rank 1 is the slow replica
        ms = bench.max_over_ranks(local, world, "cpu")
        rate = bench.job_rate(1e9, ms, world)
        env = bench.dist_env()
        # the reference arm: only rank 0 prints its line (the run itself is skipped here
        # for rank 0 by a zero-step budget, so the test stays short)
        buf = io.StringIO()
        if rank != 0:
            with contextlib.redirect_stdout(buf):
                bench.run_reference(type("A", (), {"steps": 0, "warmup": 0, "cpu_seconds": 0.0, "gpus": world})())
        out.put((rank, ms, rate, env, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_count_all_units():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate, env, printed in res:
        assert ms == 15.0                              # max over ranks, on every rank
        assert abs(rate - 2 * 1e9 / 15e-3 / 1e9) < 1e-9  # both replicas' units over the job time
        assert env == (rank, world, rank)
        if rank == 1:
            assert printed == ""                       # rank 1 of the reference arm prints nothing


def test_single_process_needs_no_collective():
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_rate(2e9, 1000.0, 1) == 2.0
