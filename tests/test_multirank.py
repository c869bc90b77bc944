"""The multi-rank bench path on CPU: two gloo ranks (one independent lattice
each, no data-path collective) agree on the slowest rank's time, and the job's
throughput is world x per-rank units / that time (weak scaling)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = 1.0 + 0.5 * rank                       # rank 1 is the slow one
    m = bench.max_over_ranks(t, dist, device="cpu")
    dist.barrier()
    out[rank] = (m, bench.weak_scaling_value(100.0, world, m))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
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
    assert out[0] == out[1] == (1.5, 2 * 100.0 / 1.5)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.25, None) == 3.25
    assert bench.weak_scaling_value(10.0, 1, 2.0) == 5.0
