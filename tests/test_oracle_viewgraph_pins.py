"""Pins of the oracle's viewgraph estimation (Section 3, Viewgraph Estimation: the share of a
view's pixels whose round trip i -> j -> i returns within tau pixels) on configurations with
closed forms: identical views, a camera translated over a fronto-parallel plane (a pure
disparity shift), a wrong target depth, a camera facing away, and invalid depth."""
import math

import numpy as np
import pytest

import oracle

W, H, F = 64, 48, 50.0
K1 = [F, F, (W - 1) / 2, (H - 1) / 2]


def two_views(b=0.0, d=5.0, zj_scale=1.0, rot_j=None):
    """View 0 at the origin, view 1 translated by b along x (camera centre at +b), both
    looking down +z at a plane z = d."""
    T0 = np.eye(4)[:3].ravel()
    R1 = np.eye(3) if rot_j is None else rot_j
    C1 = np.array([b, 0.0, 0.0])
    T1 = np.concatenate([R1, (-R1 @ C1)[:, None]], axis=1).ravel()
    Z0 = np.full((H, W), d, np.float32)
    Z1 = np.full((H, W), d * zj_scale, np.float32)
    return [W, W], [H, H], [K1, K1], np.stack([T0, T1]), [Z0, Z1]


def grid_fraction(keep_x, stride):
    xs = np.arange(0, W, stride)
    return np.mean([keep_x(x) for x in xs])


def test_identical_views_return_exactly():
    f = oracle.viewgraph(*two_views(b=0.0), stride=3, tau=1e-6)
    assert f[0, 1] == 1.0 and f[1, 0] == 1.0 and f[0, 0] == 0.0


@pytest.mark.parametrize("stride", [1, 4])
def test_disparity_shift_over_a_plane(stride):
    b, d = 0.8, 5.0
    s = F * b / d  # 8 px: a point at pixel x of view 0 is at x - 8 in view 1
    f = oracle.viewgraph(*two_views(b=b, d=d), stride=stride, tau=3.0)
    assert f[0, 1] == pytest.approx(grid_fraction(lambda x: x - s >= 0, stride), abs=1e-12)
    assert f[1, 0] == pytest.approx(grid_fraction(lambda x: x + s <= W - 1, stride), abs=1e-12)


def test_wrong_target_depth_breaks_the_round_trip():
    # view 1 believes the plane twice as far: the return lands s / 2 = 10.25 px off (a
    # disparity off the integers keeps every grid column away from the image border)
    b, d = 2.05, 5.0
    f = oracle.viewgraph(*two_views(b=b, d=d, zj_scale=2.0), stride=2, tau=3.0)
    assert f[0, 1] == 0.0
    # with a tolerance above the error every in-bounds pixel passes
    s = F * b / d
    f2 = oracle.viewgraph(*two_views(b=b, d=d, zj_scale=2.0), stride=2, tau=s / 2 + 0.5)
    assert f2[0, 1] == pytest.approx(grid_fraction(lambda x: x - s >= 0, 2), abs=1e-12)


def test_camera_facing_away_and_invalid_depth():
    Ry = np.array([[math.cos(math.pi), 0, math.sin(math.pi)], [0, 1, 0], [-math.sin(math.pi), 0, math.cos(math.pi)]])
    f = oracle.viewgraph(*two_views(b=0.0, rot_j=Ry), stride=2, tau=3.0)
    assert f[0, 1] == 0.0 and f[1, 0] == 0.0
    Wl, Hl, Kl, T, Z = two_views(b=0.0)
    Z[0][:, : W // 2] = 0.0       # no depth on the left half: those pixels do not count
    Z[0][0, W - 1] = np.nan
    f = oracle.viewgraph(Wl, Hl, Kl, T, Z, stride=1, tau=1e-6)
    assert f[0, 1] == 1.0
    Z[0][:] = 0.0
    assert oracle.viewgraph(Wl, Hl, Kl, T, Z, stride=1, tau=1e-6)[0, 1] == 0.0


def test_pairs_need_both_directions():
    frac = np.array([[0, 0.2, 0.5], [0.1, 0, 0.3], [0.6, 0.3, 0]])
    assert oracle.viewgraph_pairs(frac, 0.125).tolist() == [[0, 2], [1, 2], [2, 0], [2, 1]]
