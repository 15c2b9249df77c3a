"""Multi-GPU bookkeeping of bench.py on CPU (gloo, world size 2).

The path runs as independent replicas (one problem per GPU, no data-path
collective): the job time is the maximum over ranks and the job value is
all ranks' particles over that time.  These checks need no GPU.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.job_time(10.0 + 5.0 * rank, dist)  # rank 1 is the slow one
    out[rank] = (t, bench.job_value(1000, world, t))
    dist.destroy_process_group()


def test_job_time_is_max_over_ranks_and_value_aggregates():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    assert res[0][1] == pytest.approx(2 * 1000 / 15e-3)


def test_single_process_needs_no_collective():
    import bench
    assert bench.job_time(12.5, None) == 12.5
    assert bench.job_value(2097152, 1, 44.0) == pytest.approx(2097152 / 0.044)
