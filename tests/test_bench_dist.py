"""CPU test of the benchmark's multi-rank logic with two gloo ranks: the
timed region's duration is the slowest rank's, and the whole-job rate is
all ranks' units over that time (independent replicas, no data exchange)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t = bench.max_over_ranks(1.5 + rank, world)
    out[rank] = (t, bench.job_rate(100, world, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_and_rate():
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == out[1] == (2.5, 200 / 2.5)


def test_single_rank_is_identity():
    import bench

    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.job_rate(10, 1, 2.0) == pytest.approx(5.0)
