"""The benchmark's whole-job aggregation across ranks (units summed, the slowest rank's time),
run as two gloo ranks on the CPU: the path `bench.py --gpus N` takes under torchrun, where
every rank runs an independent replica and no collective touches the data path."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units = 1000 * (rank + 1)          # ranks may process different amounts
    ms = 10.0 + 5.0 * rank             # and finish at different times
    q.put((rank, bench.job_throughput(units, ms)))
    dist.destroy_process_group()


def test_two_rank_throughput_is_total_units_over_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        value, ms = out[r]
        assert ms == 15.0
        assert value == pytest.approx(3000 / 15e-3)


def test_single_process_throughput():
    import bench
    assert bench.job_throughput(500, 2.0) == (500 / 2e-3, 2.0)
