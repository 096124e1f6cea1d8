"""The N > 1 bench path: independent replicas, one per rank, combined by the
slowest rank's time (max all-reduce), tested with world-size-2 gloo ranks on
the CPU. The single-box path does not shard (no halo exchange is built); the
batch path shards by box with no exchange."""
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 if rank == 0 else 250.0  # rank 1 is the slow one
    value, ms = bench.combine_ranks(local_ms, 1000, 10, dist, device="cpu")
    q.put((rank, value, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_by_the_slowest():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms in out:
        assert ms == 250.0
        assert value == pytest.approx(2 * 1000 * 10 / 0.25)


def test_single_rank_needs_no_process_group():
    import bench
    value, ms = bench.combine_ranks(50.0, 400, 5, None, device="cpu")
    assert ms == 50.0 and value == pytest.approx(400 * 5 / 0.05)
