"""Pins of the oracle's optimisation schedule (Section 3, Optimization Schedule): the per-view
rotation and translation-direction changes in degrees against rotations of known angle, the
95th percentile against the numerical library's, and the dual-phase rule on hand-made
sequences of theta_95."""
import math

import numpy as np
import pytest

import oracle
from tests.test_oracle_pins import pose4


def test_pose_change_of_known_rotations_and_translations():
    rng = np.random.default_rng(1)
    n = 9
    T0 = np.zeros((n, 12))
    T1 = np.zeros((n, 12))
    angles = rng.uniform(1e-3, 2.5, n)
    tangles = rng.uniform(0.0, math.pi, n)
    for v in range(n):
        A = pose4(oracle.se3_exp(np.concatenate([rng.normal(size=3), rng.normal(size=3)])))
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        E = pose4(oracle.se3_exp(np.concatenate([[0, 0, 0], angles[v] * ax])))
        Bm = E @ A
        # translations with a known angle between them, independent lengths
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        w = np.cross(u, rng.normal(size=3))
        w /= np.linalg.norm(w)
        A[:3, 3] = 2.0 * u
        Bm[:3, 3] = 5.0 * (math.cos(tangles[v]) * u + math.sin(tangles[v]) * w)
        T0[v], T1[v] = A[:3].ravel(), Bm[:3].ravel()
    dR, dt = oracle.pose_change(T0, T1)
    assert np.allclose(dR, np.degrees(angles), rtol=1e-9, atol=1e-9)
    assert np.allclose(dt, np.degrees(tangles), rtol=1e-9, atol=1e-7)
    # no change, and a zero translation
    z = T0.copy()
    z[0, [3, 7, 11]] = 0.0
    dR0, dt0 = oracle.pose_change(z, z)
    # arccos near 1 turns a trace rounding of a few ulps (~4e-16) into ~2e-8 rad = ~1e-6 degrees
    assert np.all(dR0 < 1e-5) and np.all(dt0 < 1e-5) and dt0[0] == 0.0


@pytest.mark.parametrize("n", [1, 2, 7, 20, 101])
def test_percentile_matches_library(n):
    x = np.random.default_rng(n).exponential(size=n)
    for q in (0.0, 50.0, 95.0, 100.0):
        assert oracle.percentile(x, q) == pytest.approx(np.percentile(x, q), rel=1e-15, abs=1e-15)


def test_theta95_is_the_larger_percentile():
    rng = np.random.default_rng(4)
    T0 = np.stack([oracle.se3_exp(rng.normal(size=6)) for _ in range(40)])
    T1 = np.stack([(pose4(oracle.se3_exp(rng.normal(0, 0.01, 6))) @ pose4(t))[:3].ravel() for t in T0])
    dR, dt = oracle.pose_change(T0, T1)
    assert oracle.theta95(T0, T1) == max(np.percentile(dR, 95), np.percentile(dt, 95))


def test_dual_phase_rule():
    eps1, w1, eps2, w2 = 1.0, 3, 0.1, 3
    seq = [5, 0.5, 0.5, 0.5, 0.05, 0.05, 1, 0.05, 0.05, 0.05, 0.05]
    assert oracle.converge_run(seq, eps1, w1, eps2, w2) == [1, 1, 1, 2, 2, 2, 2, 2, 2, 3, 3]
    # a reset in phase 1: the window restarts
    assert oracle.converge_run([0.5, 0.5, 2, 0.5, 0.5, 0.5], eps1, w1, eps2, w2) == [1, 1, 1, 1, 1, 2]
    # equality with the threshold does not count as below it
    assert oracle.converge_run([1.0] * 5, eps1, w1, eps2, w2) == [1] * 5
