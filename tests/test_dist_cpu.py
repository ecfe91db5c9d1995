"""Multi-rank plumbing of bench.py on CPU (gloo, world size 2): ranks build
independent replicas, so the only cross-rank steps are the barrier and the
max over ranks of the step time."""
import os
import socket

import torch.multiprocessing as mp


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
    r, local, ws, pg = bench.dist()
    assert (r, ws) == (rank, world)
    bench.barrier(pg)
    m = bench.max_over_ranks(pg, 10.0 + rank)
    out[rank] = m
    pg.destroy_process_group()


def test_two_rank_max_over_ranks():
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    assert dict(out) == {0: 11.0, 1: 11.0}
