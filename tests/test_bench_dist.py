"""bench.py's multi-rank timing (one process per GPU, replicas): the job time is the slowest
rank's, agreed over torch.distributed.  Checked with two gloo ranks on the CPU."""
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


def _rank(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                      LOCAL_RANK=str(rank), WF_BENCH_GLOO="1")
    import bench
    ws, r, local = bench.dist_init()
    assert (ws, r, local) == (2, rank, rank)
    t = bench.barrier_max(ws, 1.5 + rank)          # rank 1 is the slow one
    bench.barrier(ws)
    out[rank] = t
    dist.destroy_process_group()


def test_slowest_rank_time_over_two_gloo_ranks():
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(_free_port(), out), nprocs=2, join=True)
    assert out[0] == out[1] == 2.5
