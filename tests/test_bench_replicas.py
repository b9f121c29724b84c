"""The multi-process path of bench.py on CPU (gloo, two ranks): replicas, no
collective in the data path; the job's time is the slowest rank's and its
V-cycles the sum over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seconds = [1.5, 2.25][rank]
    cycles = [19, 21][rank]
    out[rank] = bench.aggregate_over_ranks(seconds, cycles, world, torch.device("cpu"))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_report_slowest_time_and_summed_cycles():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (2.25, 40)


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate_over_ranks(1.25, 17, 1) == (1.25, 17)
