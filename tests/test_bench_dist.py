"""The multi-GPU bench path on CPU: two gloo ranks, host logic only.

Multi-GPU runs are independent replicas; the only cross-rank steps are the
barrier and the reductions of the timing, checked here with world size 2.
"""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import importlib.util
    import sys

    import torch.distributed as dist

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    spec = importlib.util.spec_from_file_location("bench", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    ws, r, local, pg = bench._dist()
    assert (ws, r, local) == (world, rank, rank)
    bench._barrier(pg)
    # rank r processed (r+1)*100 units in (r+1) seconds: sum 300 units over the slowest 2 s
    value, tmax = bench.aggregate(pg, (rank + 1) * 100.0, float(rank + 1))
    q.put((rank, value, tmax))
    dist.destroy_process_group()


def test_replica_aggregation_over_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, value, tmax in got:
        assert tmax == 2.0
        assert value == pytest.approx(150.0)


def test_single_process_aggregation_is_identity():
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    assert bench.aggregate(None, 10.0, 4.0) == (2.5, 4.0)
