"""The multi-rank plumbing of bench.py (replicas, barrier, max over ranks) on CPU
with the gloo backend and world size 2."""
import os
import socket

import pytest
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    assert bench.dist_env() == (ws, rank, rank)
    bench.barrier(ws)
    m = bench.max_over_ranks(ws, 10.0 + 5.0 * rank)  # rank 1 is the slow replica
    bench.barrier(ws)
    dist.destroy_process_group()
    out[rank] = m


def test_max_over_ranks_world_size_2_gloo():
    ws = 2
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_rank_main, args=(ws, _free_port(), out), nprocs=ws, join=True)
    assert dict(out) == {0: 15.0, 1: 15.0}


def test_single_rank_env_defaults(monkeypatch):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (1, 0, 0)
    assert bench.max_over_ranks(1, 3.5) == 3.5
