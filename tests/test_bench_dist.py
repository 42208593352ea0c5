"""The multi-GPU form of the benchmark (independent replicas, one per rank):
the step time is the maximum over ranks and the value the work of all ranks.
Exercised with two gloo ranks on CPU."""
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


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms, e2e = [10.0, 12.5][rank], [11.0, 13.0][rank]
    res = bench.combine_ranks(ms, e2e, 1000, world, dist, "cpu")
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_reduction():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        ms, e2e, value, e2e_value = out[r]
        assert ms == 12.5 and e2e == 13.0
        assert value == pytest.approx(2 * 5 * 1000 / 12.5e-3)
        assert e2e_value == pytest.approx(2 * 5 * 1000 / 13.0e-3)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    ms, e2e, value, e2e_value = bench.combine_ranks(8.0, 9.0, 4194304, 1)
    assert (ms, e2e) == (8.0, 9.0)
    assert value == pytest.approx(5 * 4194304 / 8.0e-3)
