"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The path shards by parameter vector (independent units, no data-path
collective); the only cross-rank step is taking the slowest rank's timed
region.  Each rank reports a different duration and every rank must see the
maximum, and each rank draws different parameter vectors.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2607_02749_gb300 import workloads as wl

    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    th = wl.thetas(6, 1, 2, seed=1 + rank)
    out[rank] = (ms, float(th.sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_per_rank_inputs():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    assert res[0][1] != res[1][1]


def test_single_process_is_identity():
    import bench

    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
