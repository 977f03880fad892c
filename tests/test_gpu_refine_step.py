"""The refinement optimiser inside the GPU step (Algorithm 2 with the camera and depth
modules: Adam on the poses, on gamma every step, on alpha and beta in the depth phase)
against the oracle's full refinement step.

Adam's first step from zero moments moves every parameter by a fixed amount against the sign
of its gradient, so a parameter whose gradient lies within the FP32 path's error of zero may
move either way on the two sides.  The single-step checks therefore compare parameters whose
oracle gradient is at least 1e-3 of the largest (ten times the gradient tolerance of the
evaluation tests) to the FP32 rounding of the move, and bound the others by the move's size.
alpha and beta are stored in FP32 on the device: their moves carry one rounding of the value."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import gpu_scene, oracle_maps_f32, rot_err_deg, trans_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA GPU required", allow_module_level=True)

import paper_2607_00579_gb300 as epo  # noqa: E402

B = epo._binding
LR_POSE = dict(lr_rot=2e-3, lr_trans=5e-2)
LR_F, LR_D = 1e-3, 1e-3
SIGNIF = 1e-3


@pytest.fixture(scope="module")
def ring8():
    sc = synth.make_scene(synth.RING8_128x96)
    maps = oracle_maps_f32(sc)
    return sc, maps, oracle.scene_from_synth(sc, [m.astype(np.float64) for m in maps])


def refinement(sc, seed=3, s=0.01):
    rng = np.random.default_rng(seed)
    n = sc.rec.shape[0]
    g = rng.normal(0, s, sc.n_views)
    a = (1.0 + rng.normal(0, s, n)).astype(np.float32)
    b = rng.normal(0, 5 * s, n).astype(np.float32)
    return g, a, b


def refine_step_scene(sc, maps, lr_focal=LR_F, lr_depth=LR_D, **kw):
    return gpu_scene(sc, maps, refine=1, lr_focal=lr_focal, lr_depth=lr_depth, **{**LR_POSE, **kw})


def get_ref(s, sc):
    return B.epo_get_refinement(s.handle, sc.n_views, sc.rec.shape[0])


def first_move(lr, t, b1=0.9, b2=0.999):
    """|move| of Adam's first step from zero moments at bias-correction count t."""
    return lr * ((1 - b1) / (1 - b1 ** t)) / np.sqrt((1 - b2) / (1 - b2 ** t))


def check_moves(d_gpu, d_or, grad, bound, ulp):
    sig = np.abs(grad) >= SIGNIF * np.abs(grad).max()
    assert sig.mean() > 0.5
    assert np.all(np.abs(d_gpu - d_or)[sig] <= 1e-5 * np.abs(d_or[sig]) + 2 * ulp[sig])
    assert np.all(np.abs(d_gpu) <= bound * (1 + 1e-5) + 2 * ulp)


@pytest.mark.parametrize("step0", [0, 9])
def test_one_step_matches_oracle(ring8, step0):
    sc, maps, o = ring8
    g, a, b = refinement(sc)
    s = refine_step_scene(sc, maps)
    s.set_poses(sc.T_init)
    B.epo_set_refinement(s.handle, g, a, b)
    s.set_state(step0)
    assert s.info().kernels_per_step == 5  # refine intrinsics, setup, edge, poses, depth
    s.step(1)
    Tg = s.get_poses()
    gg, ag, bg = get_ref(s, sc)
    st = o.refine_state(sc.T_init, g, a.astype(np.float64), b.astype(np.float64))
    f = o.loss_grad_full(sc.T_init, g, a.astype(np.float64), b.astype(np.float64), oracle.lambda_at(step0))
    loss_o = o.refine_step(st, sc.fixed, step0, step0 + 1, LR_F, LR_D, **LR_POSE)
    lg = np.zeros(1)
    B.epo_last_loss(s.handle, lg)
    assert lg[0] == pytest.approx(loss_o, rel=1e-5)
    # poses: every moving view's gradient components lie farther from zero than twice the FP32
    # path's gradient error (1e-4 of the largest) here, so no sign flips and the first Adam step
    # agrees to the FP32 rounding of its ratio
    G = f["grad"][~sc.fixed.astype(bool)]
    assert np.abs(G).min() >= 2e-4 * np.abs(G).max()
    assert np.abs(Tg - st["T"].reshape(Tg.shape)).max() < 1e-7
    # gamma: FP64 Adam on the FP32-path gradient
    check_moves(gg - g, st["gamma"] - g, f["grad_gamma"], first_move(LR_F, step0 + 1), np.zeros_like(g))
    # alpha, beta: the depth module's own count is step0 + 1 without the schedule
    for x0, xg, xo, gr in ((a, ag, st["alpha"], f["grad_alpha"]), (b, bg, st["beta"], f["grad_beta"])):
        ulp = np.spacing(np.abs(xg)).astype(np.float64)
        check_moves(xg.astype(np.float64) - x0, xo - x0.astype(np.float64), gr, first_move(LR_D, step0 + 1), ulp)


def test_trajectory_tracks_oracle(ring8):
    sc, maps, o = ring8
    g, a, b = refinement(sc)
    s = refine_step_scene(sc, maps)
    s.set_poses(sc.T_init)
    B.epo_set_refinement(s.handle, g, a, b)
    st = o.refine_state(sc.T_init, g, a.astype(np.float64), b.astype(np.float64))
    losses = [o.refine_step(st, sc.fixed, k, k + 1, LR_F, LR_D, **LR_POSE) for k in range(30)]
    s.step(30)
    Tg = s.get_poses()
    gg, ag, bg = get_ref(s, sc)
    # the tolerances of the pose-only 50-step comparison
    assert rot_err_deg(Tg, st["T"]).max() <= 0.01
    assert trans_err(Tg, st["T"], sc.scale).max() <= 1e-4
    assert np.abs(gg - st["gamma"]).max() <= 0.02 * np.abs(st["gamma"] - g).max()
    # depth: a parameter whose gradient hovers near zero follows its own sign sequence on
    # each side; most follow the same path
    z = sc.rec[:, 2].astype(np.float64)
    dz = np.abs((ag.astype(np.float64) - st["alpha"]) * z + (bg.astype(np.float64) - st["beta"]))
    moved = np.abs((st["alpha"] - a) * z + (st["beta"] - b))
    assert np.median(dz) <= 0.01 * np.median(moved)
    assert np.quantile(dz, 0.99) <= 0.2 * np.quantile(moved, 0.99)
    # and the run does what the oracle's does: the loss falls, the focal errors shrink
    assert losses[-1] < 0.5 * losses[0]
    assert np.abs(gg).mean() < 0.8 * np.abs(g).mean()
    assert rot_err_deg(Tg, sc.T_gt).mean() < rot_err_deg(sc.T_init, sc.T_gt).mean()


def test_focal_only_keeps_depth_and_single_pass(ring8):
    sc, maps, o = ring8
    g, a, b = refinement(sc)
    s = refine_step_scene(sc, maps, lr_depth=0.0)
    assert s.info().kernels_per_step == 4
    s.set_poses(sc.T_init)
    B.epo_set_refinement(s.handle, g, a, b)
    s.step(1)
    gg, ag, bg = get_ref(s, sc)
    assert np.array_equal(ag, a) and np.array_equal(bg, b)
    st = o.refine_state(sc.T_init, g, a.astype(np.float64), b.astype(np.float64))
    f = o.loss_grad_full(sc.T_init, g, a.astype(np.float64), b.astype(np.float64), oracle.lambda_at(0))
    o.refine_step(st, sc.fixed, 0, 0, LR_F, 0.0, **LR_POSE)
    check_moves(gg - g, st["gamma"] - g, f["grad_gamma"], first_move(LR_F, 1), np.zeros_like(g))


def test_depth_module_waits_for_phase_two(ring8):
    """With the schedule on, alpha and beta stay put through phase 1; the first depth step
    after the switch is the depth module's step 1 (a move of lr_depth against the gradient)."""
    sc, maps, o = ring8
    g, a, b = refinement(sc)
    # theta_95 is always below eps1 = 1e9: the switch comes at the end of step w1 - 1 = 2;
    # eps2 = 0: no convergence
    s = refine_step_scene(sc, maps, schedule=1, sched_eps1=1e9, sched_w1=3, sched_eps2=0.0, sched_w2=5)
    s.set_poses(sc.T_init)
    B.epo_set_refinement(s.handle, g, a, b)
    for k in range(3):
        s.step(1)
        _, ag, bg = get_ref(s, sc)
        assert np.array_equal(ag, a) and np.array_equal(bg, b), k
    _, phase, sw, _ = B.epo_get_schedule(s.handle, 1)
    assert phase[0] == 2 and sw[0] == 2
    gam, _, _ = get_ref(s, sc)
    T3 = s.get_poses()
    f = o.loss_grad_full(T3, gam, a.astype(np.float64), b.astype(np.float64), oracle.lambda_at(3))
    s.step(1)
    _, ag, bg = get_ref(s, sc)
    for x0, xg, gr in ((a, ag, f["grad_alpha"]), (b, bg, f["grad_beta"])):
        d = xg.astype(np.float64) - x0
        ulp = np.spacing(np.abs(xg)).astype(np.float64)
        sig = np.abs(gr) >= SIGNIF * np.abs(gr).max()
        assert np.all(np.abs(d[sig] + LR_D * np.sign(gr[sig])) <= 1e-5 * LR_D + 2 * ulp[sig])
        assert np.all(np.abs(d) <= LR_D * (1 + 1e-5) + 2 * ulp)


def test_refinement_step_options_checked(ring8):
    sc, maps, _ = ring8
    with pytest.raises(epo.EpoError):
        gpu_scene(sc, maps, lr_focal=1e-3)  # needs refine = 1
    with pytest.raises(epo.EpoError):
        gpu_scene(sc, maps, refine=1, lr_depth=-1.0)
    s = gpu_scene(sc, maps)
    with pytest.raises(epo.EpoError):
        B.epo_get_refinement(s.handle, sc.n_views, sc.rec.shape[0])
