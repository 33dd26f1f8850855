"""The multi-rank path of bench.py on the CPU: two ranks over gloo (the
barrier and max-over-ranks timing that torchrun replicas use on GPUs).  The
path does not shard across GPUs (one design per GPU, no collective in the
data path), so this is all that N > 1 adds."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.reduce_max(1.5 + rank, dist, "cpu")  # rank 1 is the slower replica
        out.put((rank, ms, bench.replica_value(world, 1000.0, ms)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.5, 2.5]
    # whole-job throughput: both replicas' units over the slowest time
    assert res[0][2] == pytest.approx(2 * 1000.0 / 2.5e-3)


def test_single_rank_is_unchanged():
    import bench
    assert bench.reduce_max(3.25, None, "cpu") == 3.25
    assert bench.replica_value(1, 10.0, 2.0) == pytest.approx(5000.0)
