"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): the
timed region is the slowest rank's, and the whole-job rate counts every
rank's independent workload copy."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    mine = [3.5, 7.25][rank]
    got = bench.max_over_ranks(mine, dist, "cpu")
    dist.barrier()
    q.put((rank, got, bench.whole_job_mlups(world, 349184, 200, got)))
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    assert [r[1] for r in res] == [7.25, 7.25]
    expect = 2 * 349184 * 200 / (7.25e-3) / 1e6
    assert all(abs(r[2] - expect) < 1e-9 * expect for r in res)
