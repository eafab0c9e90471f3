"""The multi-process path of bench.py on CPU: two gloo ranks (one per GPU in a real run)
time their own independent builds; the slowest rank's time counts and the whole-job rate
is world / that time (weak scaling, no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 10.0 + 7.5 * rank
    t = bench.max_over_ranks(local_ms, dist, "cpu")
    out[rank] = (t, bench.job_rate(world, t * 1e-3))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        t, rate = res[r]
        assert t == 17.5
        assert abs(rate - world / 0.0175) < 1e-9


def test_one_process_is_the_identity():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.job_rate(1, 0.5) == 2.0
