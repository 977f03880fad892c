"""The paper's pose parameterisation on the GPU (Section 3, Pose Refinement, Eq. 3:
P^s = phi(P^0 + MLP(P^0)) + [0 | delta], AdamW with warm-up and cosine decay) against the
FP64 oracle (oracle/pose_mlp.py on top of the C oracle's objective).

The MLP runs in FP32 on the device (the paper runs it in BF16), phi and the poses in FP64.
Tolerances: poses to 4e-6 of the MLP output's largest entry (a 128-term FP32 dot product per
layer); parameters after a step to the FP32 rounding of their move, except where the oracle's
gradient is below 1e-3 of its layer's largest (AdamW's first step moves a parameter by the
learning rate against the sign of its gradient, and a gradient within the FP32 path's error of
zero may take either sign): there only the size of the move is checked."""
import numpy as np
import pytest

import oracle
import oracle.pose_mlp as pm
import synth
from tests.helpers import gpu_scene, oracle_maps_f32, rot_err_deg, trans_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA GPU required", allow_module_level=True)

import paper_2607_00579_gb300 as epo  # noqa: E402

B = epo._binding
SIGNIF = 1e-3


@pytest.fixture(scope="module")
def ring8():
    sc = synth.make_scene(synth.RING8_128x96)
    maps = oracle_maps_f32(sc)
    return sc, maps, oracle.scene_from_synth(sc, [m.astype(np.float64) for m in maps])


def mlp_scene(sc, maps, theta, **kw):
    s = gpu_scene(sc, maps, pose_param=B.EPO_POSE_MLP, **kw)
    s.set_poses(sc.T_init)
    B.epo_set_pose_mlp(s.handle, theta)
    return s


def objective(o):
    return lambda T: (lambda r: (r["loss"], r["grad"]))(o.loss_grad(T, lam=oracle.lambda_at(0)))


def test_initial_poses_are_the_given_ones(ring8):
    sc, maps, _ = ring8
    s = mlp_scene(sc, maps, synth.pose_mlp_init())
    assert np.abs(s.get_poses().reshape(-1, 12) - np.asarray(sc.T_init).reshape(-1, 12)).max() < 1e-14
    assert s.info().kernels_per_step == 6


def test_forward_matches_oracle(ring8):
    sc, maps, _ = ring8
    rng = np.random.default_rng(7)
    theta = synth.pose_mlp_init(8)
    theta[-(12 * 128 + 12):] = rng.normal(0, 2e-3, 12 * 128 + 12).astype(np.float32)
    s = mlp_scene(sc, maps, theta)
    T_o, (cache, Pp, _) = pm.poses(theta.astype(np.float64), np.zeros((sc.n_views, 3)), sc.T_init)
    y = Pp.reshape(-1, 12) - np.asarray(sc.T_init).reshape(-1, 12)
    assert np.abs(y).max() > 1e-3  # the MLP moves the poses
    assert np.abs(s.get_poses().reshape(-1, 12) - T_o).max() <= 4e-6 * np.abs(y).max() + 1e-12


def test_one_step_matches_oracle(ring8):
    sc, maps, o = ring8
    theta = synth.pose_mlp_init()
    s = mlp_scene(sc, maps, theta)
    s.step(1)
    run = pm.PoseMLP(theta, sc.T_init)
    T0, cache = pm.poses(run.theta, run.delta, run.P0)
    r = o.loss_grad(T0, lam=oracle.lambda_at(0))
    gt, gd = pm.pose_backward(run.theta, cache, T0, r["grad"])
    loss_o, _ = run.step_with(objective(o))
    lg = np.zeros(1)
    B.epo_last_loss(s.handle, lg)
    assert lg[0] == pytest.approx(loss_o, rel=1e-5)
    pg, dg = B.epo_get_pose_mlp(s.handle, 1, sc.n_views)
    lr = pm.lr_at(0)
    offs = np.cumsum([0] + [o_ * i + o_ for o_, i in pm.DIMS])
    d_gpu = pg[0].astype(np.float64) - theta.astype(np.float64)
    d_orc = run.theta - theta.astype(np.float64)
    ulp = np.spacing(np.abs(pg[0])).astype(np.float64)
    for l in range(6):
        sl = slice(offs[l], offs[l + 1])
        g = gt[sl]
        if np.abs(g).max() == 0.0:  # layers behind the zero last layer: decay only
            assert np.all(np.abs(d_gpu[sl] - d_orc[sl]) <= 2 * ulp[sl] + 1e-12)
            continue
        # a quarter of the last layer feeds the third rotation column, which phi ignores, and
        # dead ReLUs give exact zeros: those parameters only decay, on both sides
        sig = np.abs(g) >= SIGNIF * np.abs(g).max()
        assert sig.sum() > 200
        zero = g == 0.0
        assert np.all(np.abs(d_gpu[sl] - d_orc[sl])[zero] <= 2 * ulp[sl][zero] + 1e-12)
        assert np.all(np.abs(d_gpu[sl] - d_orc[sl])[sig] <= 1e-4 * np.abs(d_orc[sl])[sig] + 2 * ulp[sl][sig])
        assert np.all(np.abs(d_gpu[sl]) <= lr * 1.001 + np.abs(theta[sl]) * lr * 0.01 + 2 * ulp[sl])
    sig = np.abs(gd) >= SIGNIF * np.abs(gd).max()
    assert np.all(np.abs(dg - run.delta)[sig] <= 1e-4 * np.abs(run.delta)[sig] + 1e-9)
    # the next poses: each last-layer parameter that moved the other way (a gradient within the
    # FP32 error of zero) shifts an output by 2 lr |a_5|, the rest agree to FP32 rounding
    l6 = slice(offs[5], offs[6])
    flips = int(np.sum(np.sign(d_gpu[l6]) != np.sign(d_orc[l6])))
    a5max = np.abs(cache[0][0][5]).max()
    dT = np.abs(s.get_poses().reshape(-1, 12) - run.poses()).max()
    assert dT < 1e-6 * (1.0 + pm.unit_scale(sc.T_init)) + flips * 2 * lr * a5max * pm.unit_scale(sc.T_init), (dT, flips)
    step, _, _ = s.get_state()
    assert step == 1


def oracle_from_device(s, sc, step):
    """An oracle run holding the device's parameters, offsets, moments and step (widened)."""
    pg, dg = B.epo_get_pose_mlp(s.handle, 1, sc.n_views)
    m, v, dm, dv = B.epo_get_pose_mlp_moments(s.handle, 1, sc.n_views)
    run = pm.PoseMLP(pg[0], sc.T_init)
    run.delta = dg.astype(np.float64)
    run.m, run.v = m[0].astype(np.float64), v[0].astype(np.float64)
    run.md, run.vd = dm.astype(np.float64), dv.astype(np.float64)
    run.step = step
    return run


@pytest.mark.parametrize("k", [5, 40])
def test_step_from_the_device_state_matches_oracle(ring8, k):
    """Step k + 1 taken from the state the device reached after k steps (inside the warm-up and
    after it): the poses it produces and the parameters' moves agree with the oracle's step from
    the same state.  A whole trajectory is not compared: early steps move the poses by ~1 degree
    and AdamW's nearly sign-like moves of thousands of weights amplify rounding differences."""
    sc, maps, o = ring8
    s = mlp_scene(sc, maps, synth.pose_mlp_init())
    s.step(k)
    run = oracle_from_device(s, sc, k)
    assert np.abs(run.poses() - s.get_poses().reshape(-1, 12)).max() < 1e-5 * pm.unit_scale(sc.T_init)
    th0 = run.theta.copy()
    run.step_with(lambda T: (lambda r: (r["loss"], r["grad"]))(o.loss_grad(T, lam=oracle.lambda_at(k))))
    s.step(1)
    pg, _ = B.epo_get_pose_mlp(s.handle, 1, sc.n_views)
    d_gpu, d_orc = pg[0].astype(np.float64) - th0, run.theta - th0
    lr = pm.lr_at(k)
    # every parameter moves by at most ~lr; the moves agree to a small fraction of lr
    assert np.abs(d_gpu - d_orc).max() <= 0.05 * lr, np.abs(d_gpu - d_orc).max() / lr
    assert np.sqrt(np.mean((d_gpu - d_orc) ** 2)) <= 2e-3 * lr
    dT = np.abs(s.get_poses().reshape(-1, 12) - run.poses()).max()
    assert dT <= 1e-4 * pm.unit_scale(sc.T_init), dT


def test_trajectory_improves_like_oracle(ring8):
    sc, maps, o = ring8
    theta = synth.pose_mlp_init()
    s = mlp_scene(sc, maps, theta)
    run = pm.PoseMLP(theta, sc.T_init)
    f = lambda T, k: (lambda r: (r["loss"], r["grad"]))(o.loss_grad(T, lam=oracle.lambda_at(k)))
    losses = [run.step_with(lambda T: f(T, k))[0] for k in range(30)]
    s.step(29)
    lg = np.zeros(1)
    B.epo_last_loss(s.handle, lg)
    s.step(1)
    Tg = s.get_poses()
    assert losses[-1] < 0.7 * losses[0]
    assert lg[0] < 0.7 * losses[0] and abs(lg[0] - losses[-2]) <= 0.15 * losses[-2]
    assert rot_err_deg(Tg, sc.T_gt).mean() < rot_err_deg(sc.T_init, sc.T_gt).mean()
    assert rot_err_deg(run.poses(), sc.T_gt).mean() < rot_err_deg(sc.T_init, sc.T_gt).mean()


def test_schedule_reads_the_mlp_pose_changes(ring8):
    sc, maps, _ = ring8
    s = mlp_scene(sc, maps, synth.pose_mlp_init(), schedule=1, sched_eps1=0.0, sched_eps2=0.0)
    T_prev = s.get_poses()
    s.step(3)  # the learning rate grows over the warm-up: the poses move every step
    T_a = s.get_poses()
    s.step(1)
    T_b = s.get_poses()
    th, phase, _, _ = B.epo_get_schedule(s.handle, 1)
    assert th[0] == pytest.approx(oracle.theta95(T_a, T_b), rel=1e-6, abs=1e-9)
    assert th[0] > 0 and phase[0] == 1
    assert np.abs(T_b - T_prev).max() > 0


def test_pose_mlp_options_checked(ring8):
    sc, maps, _ = ring8
    with pytest.raises(epo.EpoError):
        gpu_scene(sc, maps, pose_param=7)
    with pytest.raises(epo.EpoError):
        gpu_scene(sc, maps, pose_param=B.EPO_POSE_MLP, mlp_eps=0.0)
    p = gpu_scene(sc, maps)
    with pytest.raises(epo.EpoError):
        B.epo_set_pose_mlp(p.handle, synth.pose_mlp_init())
    s = gpu_scene(sc, maps, pose_param=B.EPO_POSE_MLP)
    bad = synth.pose_mlp_init()
    bad[5] = np.nan
    with pytest.raises(epo.EpoError):
        B.epo_set_pose_mlp(s.handle, bad)
