"""Focal and depth refinement on the GPU (Section 3, Eqs. 4-5: f = f0 (1 + gamma) per view,
z = z0 alpha + beta per edge pixel) against the FP64 oracle.

The oracle sees the same stored values: the records and maps the GPU holds, gamma in FP64,
alpha and beta rounded to FP32 as the GPU stores them.  Tolerances: loss 1e-5 relative and
pose gradient 1e-4 of max ||g_i|| (the FP32 path, as in the pose-only tests); the focal
gradient 1e-4 of its largest entry; the per-record depth gradients 1e-4 of their largest
entry (each is a short sum over the record's pairs of FP32 terms)."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import gpu_scene, grad_rel_err, oracle_maps_f32
from tests.test_gpu_parity import check_against_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA GPU required", allow_module_level=True)

import paper_2607_00579_gb300 as epo  # noqa: E402

B = epo._binding
GAMMA_RTOL = 1e-4
DEPTH_RTOL = 1e-4


@pytest.fixture(scope="module")
def ring8():
    sc = synth.make_scene(synth.RING8_128x96)
    return sc, oracle_maps_f32(sc)


def refinement(sc, seed=3, s=0.01):
    rng = np.random.default_rng(seed)
    n = sc.rec.shape[0]
    g = rng.normal(0, s, sc.n_views)
    a = (1.0 + rng.normal(0, s, n)).astype(np.float32)
    b = rng.normal(0, 5 * s, n).astype(np.float32)
    return g, a, b


def refined_oracle(sc, maps, g, a, b):
    """The oracle on the refined inputs (for the pose-only checks with their flip allowances)
    and the oracle's refinement objective (for the focal and depth gradients)."""
    maps64 = [m.astype(np.float64) for m in maps]
    K = sc.K.copy()
    K[:, 0] *= 1.0 + g
    K[:, 1] *= 1.0 + g
    rec = sc.rec.astype(np.float64).copy()
    rec[:, 2] = rec[:, 2] * a.astype(np.float64) + b.astype(np.float64)
    o_ref = oracle.OracleScene(sc.W, sc.H, K, sc.rec_off, rec, maps64, sc.pairs)
    o_full = oracle.scene_from_synth(sc, maps64)
    return o_ref, o_full


def refine_scene(sc, maps, **kw):
    return gpu_scene(sc, maps, refine=1, **kw)


def run_refine(s, sc):
    i = s.info()
    return B.epo_refine_loss_and_grad(s.handle, i.n_scenes, i.n_views, i.n_records)


def check_refined(sc, maps, T, g, a, b, loss, grad, gg, ga, gb, lam=10.0):
    o_ref, o_full = refined_oracle(sc, maps, g, a, b)
    r = o_ref.loss_grad(T, lam=lam)
    check_against_oracle(loss[0], grad, r, sc.pairs, T, lam=lam)
    f = o_full.loss_grad_full(T, g, a, b, lam)
    assert f["loss"] == pytest.approx(r["loss"], rel=1e-14)
    assert np.abs(gg - f["grad_gamma"]).max() <= GAMMA_RTOL * np.abs(f["grad_gamma"]).max()
    for got, want in ((ga, f["grad_alpha"]), (gb, f["grad_beta"])):
        assert np.abs(got - want).max() <= DEPTH_RTOL * np.abs(want).max()
    return f


def test_identity_refinement_equals_pose_only(ring8):
    sc, maps = ring8
    s = refine_scene(sc, maps)
    s.set_poses(sc.T_init)
    loss, grad, gg, ga, gb = run_refine(s, sc)
    p = gpu_scene(sc, maps)
    p.set_poses(sc.T_init)
    l0, g0 = p.loss_and_grad()
    # a different kernel: its rounding bound is wider (8u |X|_1 for the refined lift against
    # 6u), so a few more samples take the exact path and their FP32 terms change by ~1e-7
    # of themselves; the oracle comparison below is the one with the stated tolerances
    assert loss[0] == pytest.approx(l0[0], rel=1e-7)
    assert grad_rel_err(grad, g0) < 1e-6
    n = sc.rec.shape[0]
    check_refined(sc, maps, sc.T_init, np.zeros(sc.n_views), np.ones(n, np.float32), np.zeros(n, np.float32),
                  loss, grad, gg, ga, gb)


@pytest.mark.parametrize("gather", [epo.EPO_GATHER_LDG, epo.EPO_GATHER_TEX])
def test_refined_loss_and_all_gradients_match_oracle(ring8, gather):
    sc, maps = ring8
    g, a, b = refinement(sc)
    s = refine_scene(sc, maps, gather=gather)
    s.set_poses(sc.T_init)
    B.epo_set_refinement(s.handle, g, a, b)
    loss, grad, gg, ga, gb = run_refine(s, sc)
    check_refined(sc, maps, sc.T_init, g, a, b, loss, grad, gg, ga, gb)
    # the fused step's evaluation (pose and focal sums in one pass) gives the same loss and pose gradient
    l2, g2 = s.loss_and_grad()
    assert l2[0] == pytest.approx(loss[0], rel=1e-12) and grad_rel_err(g2, grad) < 1e-9


def test_refined_full_size_ring32():
    sc = synth.make_scene(synth.RING32_518x392)
    maps = oracle_maps_f32(sc)
    g, a, b = refinement(sc, seed=5, s=0.005)
    s = refine_scene(sc, maps)
    s.set_poses(sc.T_init)
    B.epo_set_refinement(s.handle, g, a, b)
    loss, grad, gg, ga, gb = run_refine(s, sc)
    check_refined(sc, maps, sc.T_init, g, a, b, loss, grad, gg, ga, gb)


def test_refine_scene_steps_like_pose_only_scene(ring8):
    """The same objective through the refine kernels and the pose-only kernels.  A pose-only
    scene lifts its records once, in FP64 rounded to FP32; a refine scene lifts them every step
    in FP32 (its intrinsics and depths change): the two lifted points differ by a few roundings
    (at most ~5u relative per component), so loss and gradient agree to FP32 rounding, and
    after 10 Adam steps the poses agree to the amplified rounding of every sample."""
    sc, maps = ring8
    s = refine_scene(sc, maps)
    p = gpu_scene(sc, maps)
    for h in (s, p):
        h.set_poses(sc.T_init)
    ls, gs = s.loss_and_grad()
    lp, gp = p.loss_and_grad()
    assert ls[0] == pytest.approx(lp[0], rel=1e-6) and grad_rel_err(gs, gp) < 1e-5
    for h in (s, p):
        h.step(10)
    assert np.abs(s.get_poses() - p.get_poses()).max() < 1e-5
    assert s.info().kernels_per_step == 4


def test_refinement_argument_checks(ring8):
    sc, maps = ring8
    p = gpu_scene(sc, maps)
    with pytest.raises(epo.EpoError) as e:
        B.epo_set_refinement(p.handle)
    assert e.value.status == B.EPO_ERR_INVALID_ARG
    s = refine_scene(sc, maps)
    with pytest.raises(epo.EpoError):
        B.epo_set_refinement(s.handle, np.full(sc.n_views, -1.0))
    with pytest.raises(epo.EpoError):
        refine_scene(sc, maps, records_per_thread=4)
