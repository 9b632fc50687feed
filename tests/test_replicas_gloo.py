"""The multi-process path of bench.py (replicas only): two gloo ranks on the CPU, each with
its own elapsed time; the whole-job throughput counts every rank's units over the slowest
rank's time, and all ranks agree on it."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import importlib.util
    here = os.path.dirname(os.path.abspath(__file__))
    spec = importlib.util.spec_from_file_location("bench", os.path.join(here, "..", "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        value, slowest = bench.replica_throughput(100.0 + 50.0 * rank, 8, dist, "cpu")
        q.put((rank, value, slowest))
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_max_over_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, slowest in out:
        assert slowest == 150.0
        assert abs(value - 8 * 2 / 0.150) < 1e-9


def test_single_process_has_no_collective():
    import importlib.util
    here = os.path.dirname(os.path.abspath(__file__))
    spec = importlib.util.spec_from_file_location("bench", os.path.join(here, "..", "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    value, slowest = bench.replica_throughput(200.0, 8)
    assert slowest == 200.0 and abs(value - 40.0) < 1e-12
