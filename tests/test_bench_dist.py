"""The multi-rank host logic of bench.py (one replica per GPU, N > 1): the
whole-job rate is the units of all ranks over the slowest rank's time, the
same on every rank.  World size 2 over gloo on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE="2")
    dist.init_process_group("gloo", rank=rank, world_size=2)
    import bench
    # rank 1 is the slow one: 3 s for 20 units; rank 0 takes 1 s for 10
    rate, tmax = bench.job_rate(1.0 + 2.0 * rank, 10.0 * (rank + 1))
    dist.barrier()
    out[rank] = (rate, tmax)
    dist.destroy_process_group()


def test_job_rate_is_total_units_over_slowest_rank():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        rate, tmax = res[rank]
        assert tmax == pytest.approx(3.0)
        assert rate == pytest.approx(30.0 / 3.0)


def test_job_rate_single_process_is_local_rate():
    import bench
    assert bench.job_rate(2.0, 10.0) == (5.0, 2.0)
