"""Pins of the pose-parameterisation oracle (Section 3, Pose Refinement, Eq. 3; Implementation
Details for AdamW and the learning-rate schedule) against facts outside its own arithmetic:
Gram-Schmidt returns rotations and leaves rotations unchanged; the zero-initialised last layer
makes the first poses the initial ones (the paper's neutral first iteration); central
differences of the MLP, of Gram-Schmidt and of the whole chain from the parameters through the
poses to the C oracle's objective; the schedule's shape; AdamW's first step."""
import numpy as np
import pytest

import oracle
import oracle.pose_mlp as pm
import synth


def rand_rot(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def test_gram_schmidt_returns_rotations_and_fixes_them():
    rng = np.random.default_rng(0)
    for _ in range(20):
        R = pm.gram_schmidt(rng.normal(size=3), rng.normal(size=3))
        assert np.allclose(R.T @ R, np.eye(3), atol=1e-14) and np.linalg.det(R) == pytest.approx(1.0, abs=1e-14)
        Q = rand_rot(rng)
        assert np.allclose(pm.gram_schmidt(Q[:, 0], Q[:, 1]), Q, atol=1e-14)
        # invariant to scaling a1 and to adding a multiple of a1 to a2
        a1, a2 = rng.normal(size=3), rng.normal(size=3)
        assert np.allclose(pm.gram_schmidt(3.0 * a1, a2 - 0.7 * a1), pm.gram_schmidt(a1, a2), atol=1e-13)


def test_gram_schmidt_vjp_matches_central_differences():
    rng = np.random.default_rng(1)
    a1, a2, dR = rng.normal(size=3), rng.normal(size=3), rng.normal(size=(3, 3))
    g1, g2 = pm.gram_schmidt_vjp(a1, a2, dR)
    h = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        f1 = (np.sum(dR * pm.gram_schmidt(a1 + e, a2)) - np.sum(dR * pm.gram_schmidt(a1 - e, a2))) / (2 * h)
        f2 = (np.sum(dR * pm.gram_schmidt(a1, a2 + e)) - np.sum(dR * pm.gram_schmidt(a1, a2 - e))) / (2 * h)
        assert g1[k] == pytest.approx(f1, rel=1e-7, abs=1e-9)
        assert g2[k] == pytest.approx(f2, rel=1e-7, abs=1e-9)


def test_mlp_backward_matches_central_differences():
    rng = np.random.default_rng(2)
    theta = synth.pose_mlp_init(3).astype(np.float64)
    theta[-(12 * 128 + 12):] = rng.normal(0, 0.05, 12 * 128 + 12)  # a non-zero last layer
    x = rng.normal(size=(5, 12))
    c = rng.normal(size=(5, 12))
    y, cache = pm.mlp_forward(theta, x)
    g, dx = pm.mlp_backward(theta, cache, c)
    f = lambda th, xx: np.sum(c * pm.mlp_forward(th, xx)[0])
    # a few parameters of every layer, and the input
    offs = np.cumsum([0] + [o * i + o for o, i in pm.DIMS])
    h = 1e-6
    for l in range(6):
        for k in rng.integers(offs[l], offs[l + 1], 4):
            e = np.zeros_like(theta)
            e[k] = h
            assert g[k] == pytest.approx((f(theta + e, x) - f(theta - e, x)) / (2 * h), rel=1e-6, abs=1e-8)
    e = np.zeros_like(x)
    e[1, 7] = h
    assert dx[1, 7] == pytest.approx((f(theta, x + e) - f(theta, x - e)) / (2 * h), rel=1e-6, abs=1e-8)
    # the skip connection carries gradient: zeroing W2..W3 leaves d/dW1 non-zero through it
    assert np.abs(g[:128 * 12]).max() > 0


def test_zero_last_layer_gives_the_initial_poses():
    sc = synth.make_scene(synth.RING8_128x96)
    theta = synth.pose_mlp_init().astype(np.float64)
    T, _ = pm.poses(theta, np.zeros((sc.n_views, 3)), sc.T_init)
    assert np.allclose(T, np.asarray(sc.T_init).reshape(-1, 12), atol=1e-12)


@pytest.fixture(scope="module")
def ring8():
    sc = synth.make_scene(synth.RING8_128x96)
    maps = [oracle.edt(e).astype(np.float32).astype(np.float64) for e in sc.edges]
    return sc, oracle.scene_from_synth(sc, maps)


def test_chain_to_parameters_matches_central_differences_of_the_objective(ring8):
    """Pins the conversion of the left-perturbation gradient to pose-entry derivatives, the
    Gram-Schmidt chain and the MLP backward in one: d L(P^s(theta, delta)) / d theta_k."""
    sc, o = ring8
    rng = np.random.default_rng(4)
    theta = synth.pose_mlp_init(5).astype(np.float64)
    theta[-(12 * 128 + 12):] = rng.normal(0, 2e-3, 12 * 128 + 12)
    delta = rng.normal(0, 0.01, (sc.n_views, 3))
    T, cache = pm.poses(theta, delta, sc.T_init)
    r = o.loss_grad(T, lam=10.0)
    gt, gd = pm.pose_backward(theta, cache, T, r["grad"])
    loss = lambda th, de: o.loss_grad(pm.poses(th, de, sc.T_init)[0], lam=10.0)["loss"]
    offs = np.cumsum([0] + [o_ * i + o_ for o_, i in pm.DIMS])
    # h small enough that no sample crosses a cell line or the border within +-h (at 1e-7 one
    # does for a last-layer weight and moves the quotient by 4e-4), large against FP64 noise
    h = 1e-8
    checked = 0
    for l in range(6):
        cand = np.arange(offs[l], offs[l + 1])
        cand = cand[np.argsort(-np.abs(gt[cand]))][:3]  # the layer's largest derivatives
        for k in cand:
            e = np.zeros_like(theta)
            e[k] = h
            fd = (loss(theta + e, delta) - loss(theta - e, delta)) / (2 * h)
            assert gt[k] == pytest.approx(fd, rel=1e-5, abs=1e-6), (l, k)
            checked += 1
    for v, c in ((1, 0), (3, 2), (6, 1)):
        e = np.zeros_like(delta)
        e[v, c] = h
        fd = (loss(theta, delta + e) - loss(theta, delta - e)) / (2 * h)
        assert gd[v, c] == pytest.approx(fd, rel=1e-5, abs=1e-6)
    assert checked == 18


def test_learning_rate_schedule_shape():
    lr = [pm.lr_at(s) for s in range(2000)]
    assert lr[0] == pytest.approx(3e-3 / 25) and lr[24] == pytest.approx(3e-3)
    assert all(b > a for a, b in zip(lr[:24], lr[1:25]))       # linear warm-up
    assert all(b < a for a, b in zip(lr[24:-1], lr[25:]))      # then decays
    assert lr[-1] == pytest.approx(0.0, abs=1e-15) and pm.lr_at(5000) == pytest.approx(0.0, abs=1e-15)
    mid = 25 - 1 + (2000 - 25) // 2
    assert pm.lr_at(mid) == pytest.approx(1.5e-3, rel=2e-3)   # a cosine is half-way at mid-span


def test_adamw_first_step():
    """From zero moments the step is lr * sign(g) after the decoupled decay p (1 - lr wd)."""
    rng = np.random.default_rng(6)
    p0, g = rng.normal(size=50), rng.normal(size=50)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    pm.adamw(p, g, m, v, 0, 1e-3, 0.01)
    # to lr eps / |g| (eps = 1e-8) and rounding
    assert np.all(np.abs(p - (p0 * (1 - 1e-5) - 1e-3 * np.sign(g))) <= 1e-3 * 1e-8 / np.abs(g) + 1e-15)


def test_pose_mlp_run_descends(ring8):
    sc, o = ring8
    run = pm.PoseMLP(synth.pose_mlp_init(), sc.T_init)
    f = lambda T: (lambda r: (r["loss"], r["grad"]))(o.loss_grad(T, lam=10.0))
    losses = [run.step_with(f)[0] for _ in range(40)]
    assert losses[-1] < 0.8 * losses[0]


def test_parameterisation_acts_on_the_unit_scale_scene():
    """Scaling the scene's translations by k scales the parameterised translations by k and
    leaves the rotations: the MLP sees (and moves) the scene at unit scale."""
    sc = synth.make_scene(synth.RING8_128x96)
    rng = np.random.default_rng(9)
    theta = synth.pose_mlp_init(10).astype(np.float64)
    theta[-(12 * 128 + 12):] = rng.normal(0, 1e-2, 12 * 128 + 12)
    delta = rng.normal(0, 0.01, (sc.n_views, 3))
    P0 = np.asarray(sc.T_init).reshape(-1, 3, 4)
    T1 = pm.poses(theta, delta, P0)[0].reshape(-1, 3, 4)
    P0k = P0.copy()
    P0k[:, :, 3] *= 7.0
    T2 = pm.poses(theta, delta, P0k)[0].reshape(-1, 3, 4)
    assert np.allclose(T2[:, :, :3], T1[:, :, :3], atol=1e-13)
    assert np.allclose(T2[:, :, 3], 7.0 * T1[:, :, 3], rtol=1e-12, atol=1e-12)
    assert pm.unit_scale(P0k) == pytest.approx(7.0 * pm.unit_scale(P0), rel=1e-12)
