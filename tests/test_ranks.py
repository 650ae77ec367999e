"""The multi-rank bench path on CPU: two gloo ranks run independent replicas;
the job's time is the slowest rank's and its work the sum of both."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as td  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank                 # rank 1 is the slow one
    pushed = 1000 * (rank + 1)
    res = bench.reduce_over_ranks(ms, pushed, 2.0 + rank, 500 * (rank + 1))
    out[rank] = res
    td.barrier()
    td.destroy_process_group()


def test_two_rank_reduction_is_max_time_and_summed_work():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        ms, pushed, e2e_s, e2e_ps = out[r]
        assert ms == 15.0 and pushed == 3000.0
        assert e2e_s == 3.0 and e2e_ps == 1500.0


def test_single_process_reduction_is_identity():
    import bench
    assert bench.reduce_over_ranks(3.0, 7, 1.5, 9) == (3.0, 7.0, 1.5, 9.0)
