"""The multi-rank logic of the benchmark on CPU (gloo, world size 2): the
whole-job throughput is the units of all ranks over the slowest rank's time,
and sharded batches give every rank its own scenes."""
import os
import socket

import numpy as np
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


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    from paper_2201_09212_gb300 import scenes
    assert bench.dist_setup() == (ws, rank, rank)
    elapsed = [2.0, 3.0][rank]
    units = [100.0, 50.0][rank]
    rate, tmax, total = bench.aggregate(dist, torch.device("cpu"), elapsed, units)
    # each rank's batch shard is its own seeded set of scenes
    b = scenes.lattice_batch(3, seed=scenes.SEED_BASE + 4 + 1000 * rank, side_range=(4, 5))
    q.put((rank, rate, tmax, total, b.meta["k"].tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
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
    out.sort()
    for rank, rate, tmax, total, _ in out:
        assert tmax == 3.0 and total == 150.0 and rate == 50.0
    assert out[0][4] != out[1][4]


def test_single_process_aggregate():
    import bench
    assert bench.aggregate(None, None, 2.0, 10.0) == (5.0, 2.0, 10.0)
