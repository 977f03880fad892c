"""Multi-rank paths on the CPU (two gloo ranks):
  * the benchmark's whole-job aggregation (units summed, the slowest rank's time), the path
    `bench.py --gpus N` takes under torchrun, where every rank runs an independent replica and
    no collective touches the data path;
  * a batch of independent scenes sharded by scene: each rank evaluates the objective of its
    own scenes with no exchange, and the shards together equal the whole batch's evaluation."""
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


def _shard_rank(rank, world, port, q):
    """One rank of a batch of independent scenes sharded by scene: the rank evaluates the
    oracle objective of its own scenes only; nothing is exchanged while it does."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np
    import oracle
    import synth
    from tests.helpers import oracle_maps_f32
    specs = _small_batch_specs()
    mine = list(range(rank, len(specs), world))
    res = {}
    for k in mine:
        sc = synth.make_scene(specs[k])
        o = oracle.scene_from_synth(sc, [m.astype(np.float64) for m in oracle_maps_f32(sc)])
        r = o.loss_grad(sc.T_init, lam=10.0)
        res[k] = (r["loss"], r["grad"])
    # the results are gathered only to be compared with the unsharded evaluation
    allres = [None] * world
    dist.all_gather_object(allres, res)
    q.put((rank, allres))
    dist.destroy_process_group()


def _small_batch_specs():
    import synth
    specs = synth.batch64_uneven_specs(n_scenes=4)
    for sp in specs:
        sp.width, sp.height, sp.n_views = 96, 72, min(sp.n_views, 6)
    return specs


def test_scene_sharded_objective_on_two_ranks_equals_the_whole_batch():
    """The batched objective is a set of independent per-scene objectives: two gloo ranks that
    each evaluate every other scene reproduce the one-process evaluation of the whole batch."""
    import numpy as np
    import oracle
    import synth
    from tests.helpers import oracle_maps_f32
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_shard_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    merged = {}
    for part in out[0]:
        merged.update(part)
    specs = _small_batch_specs()
    assert sorted(merged) == list(range(len(specs)))
    for k, sp in enumerate(specs):
        sc = synth.make_scene(sp)
        r = oracle.scene_from_synth(sc, [m.astype(np.float64) for m in oracle_maps_f32(sc)]).loss_grad(sc.T_init,
                                                                                                        lam=10.0)
        assert merged[k][0] == r["loss"]
        assert np.array_equal(merged[k][1], r["grad"])
