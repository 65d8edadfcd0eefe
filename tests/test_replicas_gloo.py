"""The multi-GPU form of the benchmark: independent replicas, one per rank
(the ensemble and single-grid workloads do not exchange data), reduced over
ranks as the job's timed region (longest rank) and total work (sum).  Run here
as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        el, ps = bench.reduce_over_ranks(1.0 + rank, 100.0 * (rank + 1), "cpu")
        wl = bench.make_workload("thermal2d", "fp32", seed_offset=rank)
        out[rank] = (el, ps, wl.seed)
    finally:
        dist.destroy_process_group()


def test_two_replicas_reduce_time_by_max_and_work_by_sum():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    assert res[0][:2] == (2.0, 300.0) and res[1][:2] == (2.0, 300.0)
    # every rank runs its own seeded problem (weak scaling)
    assert res[0][2] != res[1][2]
