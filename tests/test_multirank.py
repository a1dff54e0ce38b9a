"""Host-side logic of the multi-GPU bench (replicas, max-over-ranks timing),
exercised with world_size 2 on the gloo backend (CPU)."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    my_ms = 1000.0 * (rank + 1)            # rank 1 is the slow replica
    ms = bench.reduce_step_time(my_ms, dist, "cpu")
    out[rank] = (ms, bench.job_value(64, ws, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 2000.0
    assert res[0][1] == pytest.approx(2 * 64 / 2.0)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.reduce_step_time(123.0, None) == 123.0
    assert bench.job_value(64, 1, 1000.0) == 64.0
