"""The full 64-scene uneven batch (the benchmark's default workload: 4,305 views, 34,440 pairs,
3.2e8 evaluations per step, FP32 records and maps) against the FP64 oracle, in the launch
configuration the benchmark's autotuner picks for it (texture gather, 128-thread blocks, two
records per thread) and in the library's default one.

  * one loss + gradient evaluation: every scene's loss and gradient, and every pair's sums,
    element by element against the oracle (the parity tests' tolerances: loss 1e-5, gradient
    1e-4 of the scene's largest pose gradient, n_valid exact up to the oracle's near count);
  * one graph-captured optimisation step against the oracle's step from the same state;
  * the bounded host wait: a limit far below one step's duration runs out with
    EPO_ERR_TIMEOUT while the step completes normally, and the next calls succeed with the
    results of an uninterrupted run.

The oracle's maps are the oracle's own exact distance transform of every view's edge mask."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import oracle_maps_f32, scene_part
from tests.test_gpu_parity import check_against_oracle, oracle_of

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA GPU required", allow_module_level=True)

import paper_2607_00579_gb300 as epo  # noqa: E402

B = epo._binding
LR = dict(lr_rot=2e-3, lr_trans=2e-2)  # the benchmark's learning rates
BENCH_SCHEDULE = dict(gather=epo.EPO_GATHER_TEX, block_threads=128, records_per_thread=2)


@pytest.fixture(scope="module")
def batch64():
    specs = synth.batch64_uneven_specs()
    assert len(specs) == 64
    scenes = [synth.make_scene(sp) for sp in specs]
    maps = [oracle_maps_f32(sc) for sc in scenes]
    evals = sum(sc.evals() for sc in scenes)
    assert evals > 3e8
    T0 = np.concatenate([sc.T_init for sc in scenes])
    return scenes, maps, T0


def batch_scene(scenes, maps, **opt):
    return epo.Scene([scene_part(sc, m) for sc, m in zip(scenes, maps)], options=epo.default_options(**LR, **opt))


@pytest.fixture(scope="module")
def oracle_results(batch64):
    scenes, maps, _ = batch64
    out = []
    for sc, m in zip(scenes, maps):
        o = oracle_of(sc, m)
        out.append((o, o.loss_grad(sc.T_init, lam=10.0)))
    return out


@pytest.mark.parametrize("sched", [BENCH_SCHEDULE, {}], ids=["bench-schedule", "default-schedule"])
def test_full_batch_loss_grad_and_pair_sums_match_oracle(batch64, oracle_results, sched):
    scenes, maps, T0 = batch64
    b = batch_scene(scenes, maps, **sched)
    b.set_poses(T0)
    info = b.info()
    assert info.n_scenes == 64 and info.n_views == 4305 and info.evals_per_step > 3e8
    loss, grad = b.loss_and_grad()
    st = b.pair_stats()
    off = poff = 0
    for k, (sc, (o, r)) in enumerate(zip(scenes, oracle_results)):
        check_against_oracle(loss[k], grad[off:off + sc.n_views], r, sc.pairs, sc.T_init,
                             stats=st[poff:poff + sc.n_pairs])
        off += sc.n_views
        poff += sc.n_pairs
    queued, overflow = B.epo_fixup_stats(b.handle)
    assert 0 < queued < 0.02 * info.evals_per_step and overflow == 0


def test_full_batch_graph_step_matches_oracle_step(batch64, oracle_results):
    """Adam's first step from zero moments moves every twist component by its learning rate
    against the sign of its gradient (m_hat / sqrt(v_hat) = g / |g|), so a component whose
    oracle gradient lies within the FP32 path's gradient error (1e-4 of the scene's largest
    pose gradient) may move either way on the two sides.  Poses whose six components all lie
    beyond twice that agree to the rounding of the step; the others move by at most the
    learning rate per component, either way."""
    scenes, maps, T0 = batch64
    b = batch_scene(scenes, maps, **BENCH_SCHEDULE)
    b.set_poses(T0)
    b.step(1)
    Tg = b.get_poses()
    lg = np.zeros(64)
    B.epo_last_loss(b.handle, lg)
    lr = np.array([LR["lr_trans"]] * 3 + [LR["lr_rot"]] * 3)
    off = 0
    n_exact = 0
    for k, (sc, (o, r)) in enumerate(zip(scenes, oracle_results)):
        To, _, _, hist = o.optimize(sc.T_init, sc.fixed, 1, **LR)
        assert lg[k] == pytest.approx(hist[0], rel=1e-5)
        G = r["grad"]
        gmax = np.linalg.norm(G, axis=1).max()
        Tk = Tg[off:off + sc.n_views]
        for v in range(sc.n_views):
            if sc.fixed[v]:
                assert np.array_equal(Tk[v], sc.T_init[v])
                continue
            if np.all(np.abs(G[v]) >= 2e-4 * gmax):
                assert np.abs(Tk[v] - To[v]).max() < 1e-7, (k, v)
                n_exact += 1
            else:
                Mg = np.vstack([Tk[v].reshape(3, 4), [0, 0, 0, 1]])
                Mo = np.vstack([To[v].reshape(3, 4), [0, 0, 0, 1]])
                xi = oracle.se3_log((Mg @ np.linalg.inv(Mo))[:3].reshape(-1))
                assert np.all(np.abs(xi) <= 2 * lr * (1 + 1e-3) + 1e-9), (k, v, xi)
        off += sc.n_views
    assert n_exact > 0.5 * (4305 - 64)


def test_bounded_wait_runs_out_and_the_handle_recovers(batch64):
    scenes, maps, T0 = batch64
    b = batch_scene(scenes, maps, **BENCH_SCHEDULE)
    ref = batch_scene(scenes, maps, **BENCH_SCHEDULE)
    for h in (b, ref):
        h.set_poses(T0)
    # a step takes ~2 ms: a 1 us limit runs out while the step completes normally
    B.epo_set_wait_limit(b.handle, 1e-6)
    with pytest.raises(epo.EpoError) as e:
        b.step(1)
    assert e.value.status == B.EPO_ERR_TIMEOUT
    # with room to wait, the next call succeeds: the step ran
    B.epo_set_wait_limit(b.handle, 60.0)
    b.check()
    ref.step(1)
    assert np.abs(b.get_poses() - ref.get_poses()).max() < 1e-9
    # the host-driven step: the wait runs out again, its host outputs are not written, and
    # the step still happens
    B.epo_set_wait_limit(b.handle, 1e-6)
    T_out = np.full((4305, 12), np.nan)
    with pytest.raises(epo.EpoError) as e:
        B.epo_step_host(b.handle, None, T_out, None)
    assert e.value.status == B.EPO_ERR_TIMEOUT
    assert np.isnan(T_out).all()
    B.epo_set_wait_limit(b.handle, 60.0)
    ref.step(1)
    assert np.abs(b.get_poses() - ref.get_poses()).max() < 1e-9
    assert b.get_state()[0] == 2
    loss = np.zeros(64)
    B.epo_step_host(b.handle, None, T_out, loss)
    ref.step(1)
    assert np.abs(T_out - ref.get_poses().reshape(-1, 12)).max() < 1e-9
    lr_ = np.zeros(64)
    B.epo_last_loss(ref.handle, lr_)
    assert np.allclose(loss, lr_, rtol=1e-12, atol=0)
    # no limit (the default) also works, and a bad limit is refused
    B.epo_set_wait_limit(b.handle, 0.0)
    b.step(1)
    with pytest.raises(epo.EpoError):
        B.epo_set_wait_limit(b.handle, -1.0)
