"""Multi-rank host logic of bench.py on CPU (gloo, world_size 2).

With N GPUs every rank runs its own replica of the product (no collective on
the data path); the JSON line's time is the slowest rank's and its value the
work of all ranks over that time.  Each rank here reports a different step
time; both must see the maximum, and the whole-job value must count both
ranks' work.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 1.0 + rank          # rank 1 is the slow one
        ms = bench.reduce_max(local_ms, world, "cpu")
        out[rank] = (ms, bench.job_value(10e9, world, ms))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert sorted(res) == [0, 1]
    for ms, value in res.values():
        assert ms == pytest.approx(2.0)
        # 2 ranks x 10 GFLOP in 2 ms = 10 TFLOP/s
        assert value == pytest.approx(10.0)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max(3.5, 1, "cpu") == pytest.approx(3.5)
    assert bench.job_value(4e9, 1, 2.0) == pytest.approx(2.0)
