"""Pins of the oracle's full refinement step (Algorithm 2 with the camera and depth modules:
Adam on the poses, on gamma every step, on alpha and beta in the depth phase) against facts
outside its own update arithmetic: with zero refinement rates it is the pose-only step; Adam's
first step moves every parameter by exactly its rate against the sign of its gradient (m^ / sqrt(v^)
= sign(g)), wherever the step counter stands for the depth module once its own count restarts at 1;
the moments of two steps follow the closed form of two gradients; small steps descend."""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def ring8():
    sc = synth.make_scene(synth.RING8_128x96)
    maps = [oracle.edt(e).astype(np.float32).astype(np.float64) for e in sc.edges]
    return sc, oracle.scene_from_synth(sc, maps)


def fresh(sc, o, seed=3, s=0.01):
    rng = np.random.default_rng(seed)
    n = sc.rec.shape[0]
    return o.refine_state(sc.T_init, rng.normal(0, s, sc.n_views), 1.0 + rng.normal(0, s, n), rng.normal(0, 5 * s, n))


def test_zero_refinement_rates_give_the_pose_only_step(ring8):
    sc, o = ring8
    n = sc.rec.shape[0]
    st = o.refine_state(sc.T_init, np.zeros(sc.n_views), np.ones(n), np.zeros(n))
    loss0 = o.refine_step(st, sc.fixed, 0, 0, 0.0, 0.0)
    T1, _, _, losses = o.optimize(sc.T_init, sc.fixed, 1)
    assert np.array_equal(st["T"].reshape(-1, 3, 4), np.asarray(T1).reshape(-1, 3, 4))
    assert loss0 == losses[0]
    assert np.array_equal(st["gamma"], np.zeros(sc.n_views))
    assert np.array_equal(st["alpha"], np.ones(n)) and np.array_equal(st["beta"], np.zeros(n))


@pytest.mark.parametrize("step", [0, 7])
def test_first_adam_step_moves_each_parameter_by_its_rate(ring8, step):
    """At the first step of a module, m^ = g and v^ = g^2, so each parameter moves by the rate
    against sign(g) (to eps / |g|); the depth module counts its own steps from 1 even when the
    global step is 7, while gamma's bias factors use the global count (only step 0 is a first step)."""
    sc, o = ring8
    st = fresh(sc, o)
    g0, a0, b0 = st["gamma"].copy(), st["alpha"].copy(), st["beta"].copy()
    f = o.loss_grad_full(sc.T_init, g0, a0, b0, oracle.lambda_at(step))
    lf, ld = 3e-4, 2e-3
    o.refine_step(st, sc.fixed, step, 1, lf, ld)
    for x0, x1, g, lr in ((a0, st["alpha"], f["grad_alpha"], ld), (b0, st["beta"], f["grad_beta"], ld)):
        live = np.abs(g) > 1e-6
        assert live.sum() > 0.5 * g.size
        assert np.allclose((x1 - x0)[live], -lr * np.sign(g[live]), rtol=2e-6, atol=1e-15)  # eps / |g| <= 1e-6
        assert np.array_equal(x1[~live & (g == 0)], x0[~live & (g == 0)])
    if step == 0:
        assert np.allclose(st["gamma"] - g0, -lf * np.sign(f["grad_gamma"]), rtol=1e-9, atol=0)
    else:  # bias factors of step 8 on a fresh moment: |change| = lr (1-b1)/(1-b1^8) sqrt(1-b2^8)/sqrt(1-b2)
        k = (0.1 / (1 - 0.9 ** 8)) * np.sqrt(1 - 0.999 ** 8) / np.sqrt(0.001)
        assert np.allclose(st["gamma"] - g0, -lf * k * np.sign(f["grad_gamma"]), rtol=1e-9, atol=0)


def test_depth_module_idle_before_its_phase(ring8):
    sc, o = ring8
    st = fresh(sc, o)
    a0, b0 = st["alpha"].copy(), st["beta"].copy()
    o.refine_step(st, sc.fixed, 0, 0, 1e-3, 1e-3)
    assert np.array_equal(st["alpha"], a0) and np.array_equal(st["beta"], b0)
    assert not np.any(st["ma"]) and not np.any(st["vb"])


def test_two_steps_follow_the_closed_form_of_two_gradients(ring8):
    """After gradients g1, g2: m = 0.09 g1 + 0.1 g2, v = 0.000999 g1^2 + 0.001 g2^2, and the second
    move is lr (m / 0.19) / sqrt(v / 0.001999) against it (gradients from the pinned objective)."""
    sc, o = ring8
    st = fresh(sc, o)
    lf, ld = 1e-3, 1e-3
    f1 = o.loss_grad_full(st["T"].copy(), st["gamma"].copy(), st["alpha"].copy(), st["beta"].copy(), oracle.lambda_at(0))
    o.refine_step(st, sc.fixed, 0, 1, lf, ld)
    g1, a1, b1 = st["gamma"].copy(), st["alpha"].copy(), st["beta"].copy()
    f2 = o.loss_grad_full(st["T"].copy(), g1, a1, b1, oracle.lambda_at(1))
    o.refine_step(st, sc.fixed, 1, 2, lf, ld)
    for x1, x2, ga, gb, lr in ((g1, st["gamma"], f1["grad_gamma"], f2["grad_gamma"], lf),
                               (b1, st["beta"], f1["grad_beta"], f2["grad_beta"], ld)):
        m = 0.09 * ga + 0.1 * gb
        v = 0.000999 * ga ** 2 + 0.001 * gb ** 2
        want = -lr * (m / 0.19) / (np.sqrt(v / 0.001999) + 1e-12)
        assert np.allclose(x2 - x1, want, rtol=1e-9, atol=1e-15)


def test_small_steps_descend(ring8):
    sc, o = ring8
    st = fresh(sc, o)
    losses = [o.refine_step(st, sc.fixed, k, k + 1, 1e-4, 1e-4, lr_rot=1e-4, lr_trans=1e-3, lambda_steps=10 ** 9)
              for k in range(6)]
    assert all(b < a for a, b in zip(losses, losses[1:]))
