"""The N > 1 path of the benchmark on CPU: gloo ranks, world size 2.  Each rank runs an
independent replica; the job time is the max over ranks and the throughput counts every rank's
steps."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [4.0, 5.0][rank]
    q.put((rank, bench.aggregate(ms, world, None)))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_max_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        ms, value = out[r]
        assert ms == pytest.approx(5.0)
        assert value == pytest.approx(2 * 1000.0 / 5.0)


def test_aggregate_single_rank():
    import bench
    assert bench.aggregate(2.0, 1) == (2.0, 500.0)
