"""The benchmark's multi-rank bookkeeping with two gloo ranks on CPU.

Under torchrun every rank scores its own query batch against its own copy
of the database (independent problems, no collective on the data path);
whole-job throughput is the cells of all ranks over the slowest rank's time.
This checks that combination, and the barrier, with real process groups.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    d = bench.Dist(backend="gloo")
    d.barrier()
    local_ms = 100.0 * (rank + 1)          # rank 1 is the slow one
    local_cells = 1e12 * (rank + 1)
    t, cells, gcups = bench.combine_ranks(d, local_ms, local_cells)
    out[rank] = (t, cells, gcups)
    d.close()


def test_two_gloo_ranks_combine():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        t, cells, gcups = out[r]
        assert t == pytest.approx(200.0)
        assert cells == pytest.approx(3e12)
        assert gcups == pytest.approx(3e12 / 0.2 / 1e9)


def test_single_process_is_identity():
    import bench
    d = bench.Dist(init=False)
    assert bench.combine_ranks(d, 50.0, 1e11) == (50.0, 1e11, pytest.approx(1e11 / 0.05 / 1e9))
