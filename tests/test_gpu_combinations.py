"""The next rows combined with each other and with the precision and batching rows, against the
oracle: refinement on FP16 depth records and BF16 maps, one pose MLP per scene of a batch, and
refinement, sub-sampling and the schedule in one step graph.  Tolerances as in the single-row
tests (loss 1e-5, gradients 1e-4 of their largest entry, on the stored values)."""
import dataclasses

import numpy as np
import pytest

import oracle
import oracle.pose_mlp as pm
import synth
from tests.helpers import bf16_bits, gpu_scene, oracle_maps_f32, scene_part
from tests.test_gpu_parity import check_against_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA GPU required", allow_module_level=True)

import paper_2607_00579_gb300 as epo  # noqa: E402

B = epo._binding


def bf16_to_f32(b):
    return (np.asarray(b, dtype=np.uint32) << 16).view(np.float32)


@pytest.fixture(scope="module")
def ring8():
    sc = synth.make_scene(synth.RING8_128x96)
    return sc, oracle_maps_f32(sc)


def test_refinement_on_fp16_depth_and_bf16_maps(ring8):
    sc, maps = ring8
    rng = np.random.default_rng(11)
    n = sc.rec.shape[0]
    g = rng.normal(0, 0.01, sc.n_views)
    a = (1.0 + rng.normal(0, 0.01, n)).astype(np.float32)
    b = rng.normal(0, 0.05, n).astype(np.float32)
    s = gpu_scene(sc, [bf16_bits(m) for m in maps], rec=synth.records_f16(sc.rec), record_dtype=epo.EPO_F16,
                  map_dtype=epo.EPO_BF16, refine=1)
    s.set_poses(sc.T_init)
    B.epo_set_refinement(s.handle, g, a, b)
    loss, grad, gg, ga, gb = B.epo_refine_loss_and_grad(s.handle, 1, sc.n_views, n)
    # the oracle on the stored values: widened FP16 records, widened BF16 maps
    rec16 = synth.records_f16_widened(sc.rec)
    maps16 = [bf16_to_f32(bf16_bits(m)).astype(np.float64) for m in maps]
    o = oracle.scene_from_synth(sc, maps16, rec=rec16)
    f = o.loss_grad_full(sc.T_init, g, a.astype(np.float64), b.astype(np.float64), 10.0)
    K = sc.K.copy()
    K[:, 0] *= 1.0 + g
    K[:, 1] *= 1.0 + g
    rr = np.asarray(rec16, dtype=np.float64).copy()
    rr[:, 2] = rr[:, 2] * a.astype(np.float64) + b.astype(np.float64)
    r = oracle.OracleScene(sc.W, sc.H, K, sc.rec_off, rr, maps16, sc.pairs).loss_grad(sc.T_init, lam=10.0)
    assert f["loss"] == pytest.approx(r["loss"], rel=1e-14)
    check_against_oracle(loss[0], grad, r, sc.pairs, sc.T_init)
    assert np.abs(gg - f["grad_gamma"]).max() <= 1e-4 * np.abs(f["grad_gamma"]).max()
    for got, want in ((ga, f["grad_alpha"]), (gb, f["grad_beta"])):
        assert np.abs(got - want).max() <= 1e-4 * np.abs(want).max()


def test_one_pose_mlp_per_scene_of_a_batch():
    specs = [synth.RING8_128x96, dataclasses.replace(synth.RING8_128x96, seed=20260011, rot_noise_deg=1.5)]
    scenes = [synth.make_scene(sp) for sp in specs]
    maps = [oracle_maps_f32(x) for x in scenes]
    thetas = [synth.pose_mlp_init(20260100 + k) for k in range(2)]
    s = epo.Scene([scene_part(x, m) for x, m in zip(scenes, maps)],
                  options=epo.default_options(pose_param=B.EPO_POSE_MLP))
    s.set_poses(np.concatenate([x.T_init for x in scenes]))
    B.epo_set_pose_mlp(s.handle, np.concatenate(thetas))
    s.step(1)
    pg, dg = B.epo_get_pose_mlp(s.handle, 2, sum(x.n_views for x in scenes))
    Tg = s.get_poses().reshape(-1, 12)
    v0 = 0
    for k, (x, m) in enumerate(zip(scenes, maps)):
        o = oracle.scene_from_synth(x, [mm.astype(np.float64) for mm in m])
        run = pm.PoseMLP(thetas[k], x.T_init)
        run.step_with(lambda T: (lambda r: (r["loss"], r["grad"]))(o.loss_grad(T, lam=oracle.lambda_at(0))))
        # the first step moves each parameter by lr against its gradient's sign: the device's moves
        # agree with the oracle's wherever the oracle's move is a full step
        d_gpu = pg[k].astype(np.float64) - thetas[k].astype(np.float64)
        d_orc = run.theta - thetas[k].astype(np.float64)
        full = np.abs(d_orc) > 0.5 * pm.lr_at(0)
        assert full.sum() > 200
        assert np.mean(np.sign(d_gpu[full]) == np.sign(d_orc[full])) > 0.995
        assert np.abs(dg[v0:v0 + x.n_views] - run.delta).max() <= 1e-4 * pm.lr_at(0) + 1e-9
        assert np.abs(Tg[v0:v0 + x.n_views] - run.poses()).max() < 1e-3 * pm.unit_scale(x.T_init)
        v0 += x.n_views


def test_refinement_subsampling_and_schedule_in_one_step(ring8):
    sc, maps = ring8
    seed = 0x5EED
    s = gpu_scene(sc, maps, refine=1, lr_focal=1e-3, lr_depth=1e-3, pair_budget=24, subsample_seed=seed,
                  schedule=1, sched_eps1=1e9, sched_w1=2, sched_eps2=0.0)
    # subsample, refine intrinsics, setup, edge, poses, depth, schedule
    assert s.info().kernels_per_step == 7
    s.set_poses(sc.T_init)
    s.step(1)
    lg = np.zeros(1)
    B.epo_last_loss(s.handle, lg)
    ids = np.flatnonzero(oracle.subsample(seed, 0, sc.n_pairs, 24))
    o = oracle.OracleScene(sc.W, sc.H, sc.K, sc.rec_off, sc.rec, [m.astype(np.float64) for m in maps], sc.pairs[ids])
    assert lg[0] == pytest.approx(o.loss_grad(sc.T_init, lam=10.0)["loss"], rel=1e-5)
    s.step(4)  # phase 2 from the end of step 1: the depth module steps from step 2 on
    _, phase, sw, _ = B.epo_get_schedule(s.handle, 1)
    assert phase[0] == 2 and sw[0] == 1
    gam, al, be = B.epo_get_refinement(s.handle, sc.n_views, sc.rec.shape[0])
    assert np.abs(gam).max() > 0 and np.abs(al - 1.0).max() > 0 and np.abs(be).max() > 0
    assert np.all(np.isfinite(s.get_poses()))
