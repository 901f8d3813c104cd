"""The N > 1 path of bench.py (replicas, one process per GPU) on CPU ranks:
two gloo processes report different times; both must agree on the slowest
time and on whole-job throughput = units of all ranks / slowest time."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_ms = [12.0, 20.0][rank]
    t_max, ups = bench.aggregate_ranks(t_ms, 1000.0, world)
    out[rank] = (t_max, ups)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1]
    t_max, ups = out[0]
    assert t_max == 20.0
    assert ups == pytest.approx(2 * 1000.0 / 0.020)


def _rank_fails(rank, world, port, out):
    import datetime
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=10))
    import bench
    if rank == 1:
        out[rank] = "left"
        os._exit(3)          # a replica that dies between steps, before the aggregation
    try:
        bench.aggregate_ranks(12.0, 1000.0, world)
        out[rank] = "no error"
    except Exception as exc:  # the surviving rank learns of it from the collective
        out[rank] = "error: " + type(exc).__name__


def test_a_rank_that_dies_is_detected_by_the_others():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_fails, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert procs[1].exitcode == 3 and out[1] == "left"
    assert procs[0].exitcode == 0 and out[0].startswith("error")
