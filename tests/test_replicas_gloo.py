"""The multi-GPU path of bench.py is replicas only (independent, differently
seeded systems per rank, no data-path collective): the only cross-rank steps
are the barrier and the max over ranks of the timed region.  This runs that
logic on CPU with the gloo backend at world size 2."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    bench = _bench()
    local_ms = [12.5, 30.0][rank]  # rank 1 is the slow one
    dist.barrier()
    ms = bench.max_over_ranks(local_ms, dist, "cpu")
    value = bench.whole_job_value(world, 1024 * 1024 * 256, ms)
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        ms, value = out[r]
        assert ms == 30.0
        assert value == pytest.approx(2 * 1024 * 1024 * 256 / 0.030)


def test_single_rank_needs_no_process_group():
    bench = _bench()
    assert bench.max_over_ranks(7.0) == 7.0
    assert bench.whole_job_value(1, 1000.0, 2.0) == pytest.approx(5e5)
