"""Pins of the oracle's focal and depth refinement (Section 3, Camera Refinement and Depth
Refinement: f_i = f_i^0 (1 + gamma_i), Z = Z^0 alpha + beta per pixel) against facts
outside the oracle's own arithmetic: the reduction to the pose-only objective, the literal
brute-force loss on the refined intrinsics and depths, central differences, and the
scale gauge of the objective."""
import numpy as np
import pytest

import oracle
import synth
from oracle.brute import brute_loss
from tests.test_oracle_pins import pose4  # noqa: F401  (shared numpy helper of the pins)


@pytest.fixture(scope="module")
def ring8():
    sc = synth.make_scene(synth.RING8_128x96)
    maps = [oracle.edt(e).astype(np.float32).astype(np.float64) for e in sc.edges]
    return sc, maps, oracle.scene_from_synth(sc, maps)


def refinement(sc, seed=3, s=0.01):
    rng = np.random.default_rng(seed)
    n = sc.rec.shape[0]
    return (rng.normal(0, s, sc.n_views), 1.0 + rng.normal(0, s, n), rng.normal(0, 5 * s, n))


def test_identity_refinement_is_the_pose_objective(ring8):
    sc, maps, o = ring8
    n = sc.rec.shape[0]
    r = o.loss_grad_full(sc.T_init, np.zeros(sc.n_views), np.ones(n), np.zeros(n), 10.0)
    r0 = o.loss_grad(sc.T_init, 10.0)
    assert r["loss"] == r0["loss"]
    assert np.array_equal(r["grad"], r0["grad"])


def test_refined_loss_equals_brute_force_on_refined_inputs(ring8):
    sc, maps, o = ring8
    g, a, b = refinement(sc)
    r = o.loss_grad_full(sc.T_init, g, a, b, 10.0)
    K = sc.K.copy()
    K[:, 0] *= 1.0 + g
    K[:, 1] *= 1.0 + g
    rec = sc.rec.astype(np.float64).copy()
    rec[:, 2] = rec[:, 2] * a + b
    L = brute_loss(sc.W, sc.H, K, sc.rec_off, rec, maps, sc.pairs, sc.T_init, 10.0)
    assert r["loss"] == pytest.approx(L, rel=1e-13)


def test_focal_gradient_matches_central_differences(ring8):
    sc, maps, o = ring8
    g, a, b = refinement(sc)
    r = o.loss_grad_full(sc.T_init, g, a, b, 10.0)
    h = 1e-9
    fd = np.zeros(sc.n_views)
    for v in range(sc.n_views):
        e = np.zeros(sc.n_views)
        e[v] = h
        fd[v] = (o.loss_grad_full(sc.T_init, g + e, a, b, 10.0)["loss"]
                 - o.loss_grad_full(sc.T_init, g - e, a, b, 10.0)["loss"]) / (2 * h)
    assert np.abs(fd - r["grad_gamma"]).max() <= 1e-5 * np.abs(r["grad_gamma"]).max()


def test_depth_gradients_match_central_differences(ring8):
    sc, maps, o = ring8
    g, a, b = refinement(sc)
    r = o.loss_grad_full(sc.T_init, g, a, b, 10.0)
    rng = np.random.default_rng(8)
    ids = rng.choice(np.flatnonzero(np.abs(r["grad_beta"]) > 1e-3 * np.abs(r["grad_beta"]).max()), 24,
                     replace=False)
    h = 1e-7
    # rounding floor of a central difference of L: 4 eps |L| / (2 h) (one record moves L by
    # only ~1e-4 h, so this floor matters)
    floor = 4 * np.finfo(float).eps * abs(r["loss"]) / (2 * h)
    for k in ids:
        for name, base in (("grad_alpha", a), ("grad_beta", b)):
            hp, hm = base.copy(), base.copy()
            hp[k] += h
            hm[k] -= h
            args = (g, hp, b) if name == "grad_alpha" else (g, a, hp)
            argm = (g, hm, b) if name == "grad_alpha" else (g, a, hm)
            fd = (o.loss_grad_full(sc.T_init, *args, 10.0)["loss"]
                  - o.loss_grad_full(sc.T_init, *argm, 10.0)["loss"]) / (2 * h)
            assert fd == pytest.approx(r[name][k], rel=1e-5, abs=floor)
    # alpha scales the prior depth, beta offsets it: dL/dalpha = dL/dbeta * Z0
    assert np.allclose(r["grad_alpha"], r["grad_beta"] * sc.rec[:, 2].astype(np.float64), rtol=1e-14, atol=0)


def test_scale_gauge_identity(ring8):
    """Scaling the world by s (every translation and every depth) leaves the objective
    unchanged, so its derivative in s vanishes: sum_i t_i . dL/dt_i + sum_r z_r dL/dz_r = 0,
    with dL/dt_i the translation part of the left-perturbation gradient and dL/dz_r = dL/dbeta_r."""
    sc, maps, o = ring8
    g, a, b = refinement(sc)
    r = o.loss_grad_full(sc.T_init, g, a, b, 10.0)
    t = sc.T_init.reshape(-1, 3, 4)[:, :, 3]
    z = sc.rec[:, 2].astype(np.float64) * a + b
    terms = np.concatenate([(t * r["grad"][:, :3]).ravel(), z * r["grad_beta"]])
    assert abs(terms.sum()) <= 1e-10 * np.abs(terms).sum()
