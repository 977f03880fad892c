"""The pose kernel's rounding bound, checked on the CPU against FP32 arithmetic emulated
step by step (every product and sum rounded as the kernel rounds it) and the exact position.

The kernel takes a sample's cell, border and depth decisions in FP32 wherever the bound
    |Y_k - Y_k*| <= E = X.w + Et,  X.w = u (5 |X0| + 4 |X1| + 2 z + 2 eps_z),  Et = 4u |t|_1
    |u' - u'*|  <= t = E |1/Y3| Kb + cb
(u = 2^-24, each constant with a 1e-5 margin; Kb and cb from the target's intrinsics) shows them
to be those of the exact evaluation.  The test draws poses, intrinsics (principal points far off
centre included), depths and pixels, emulates the kernel's FP32 steps (the lift rounded from
FP64, the FMA chain with z last, a reciprocal carrying the full 2u error that rcp.approx
allows, the product and the projection FMA) and checks both inequalities on every sample whose
FP32 position lies within one pixel of the image and whose bound is at most 1/4.  The exact
values are FP64 evaluations of the same definitions (their own error, ~1e-16 relative, is far
below the 1e-5 margin)."""
import numpy as np
import pytest

U = 2.0 ** -24
MARGIN = 1.0 + 1e-5


def f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def fma32(a, b, c):
    # a*b is exact in FP64 for FP32 operands; the sum then rounds to FP64 and to FP32 (the
    # double rounding is ~2^-53 relative, far below the margin)
    return f32(a * b + c)


def rotation(axis_angle):
    """Rodrigues' formula, one rotation per row of axis-angle vectors."""
    th = np.linalg.norm(axis_angle, axis=1)
    k = axis_angle / np.maximum(th, 1e-300)[:, None]
    Kx = np.zeros((len(th), 3, 3))
    Kx[:, 0, 1], Kx[:, 0, 2], Kx[:, 1, 2] = -k[:, 2], k[:, 1], -k[:, 0]
    Kx -= Kx.transpose(0, 2, 1)
    s, c = np.sin(th)[:, None, None], np.cos(th)[:, None, None]
    return np.eye(3) + s * Kx + (1 - c) * Kx @ Kx


def bound_constants(fx, fy, cx, cy, W, H):
    """Kb and cb as the library sets them at scene creation."""
    mu = np.maximum(cx + 1.0, W - cx)
    mv = np.maximum(cy + 1.0, H - cy)
    Kb = np.maximum(fx + mu + 0.25, fy + mv + 0.25) * MARGIN
    cb = U * np.maximum(W + 4 * mu + np.abs(cx), H + 4 * mv + np.abs(cy)) * MARGIN
    return f32(Kb), f32(cb)


def draw(seed, n, off_centre):
    rng = np.random.default_rng(seed)
    W = rng.integers(64, 1024, size=n).astype(np.float64)
    H = rng.integers(48, 1024, size=n).astype(np.float64)
    fx = rng.uniform(40.0, 2500.0, size=n)
    fy = fx * rng.uniform(0.8, 1.25, size=n)
    if off_centre:
        cx = rng.uniform(-0.5, 1.5, size=n) * W
        cy = rng.uniform(-0.5, 1.5, size=n) * H
    else:
        cx, cy = (W - 1) / 2, (H - 1) / 2
    # source pixel and depth (the lift uses view i's intrinsics: drawn the same way)
    fxi = rng.uniform(40.0, 2500.0, size=n)
    fyi = fxi * rng.uniform(0.8, 1.25, size=n)
    cxi = rng.uniform(-0.5, 1.5, size=n) * W if off_centre else (W - 1) / 2
    cyi = rng.uniform(-0.5, 1.5, size=n) * H if off_centre else (H - 1) / 2
    u = f32(rng.uniform(0, W - 1))
    v = f32(rng.uniform(0, H - 1))
    z = f32(np.exp(rng.uniform(np.log(0.05), np.log(200.0), size=n)))
    # relative pose: half of the rotations small (neighbouring views), half arbitrary; a
    # translation from a hundredth to twenty scene units
    ang = rng.normal(size=(n, 3))
    ang *= np.where(rng.random(n) < 0.5, 0.3, np.pi)[:, None] / np.maximum(np.linalg.norm(ang, axis=1), 1e-12)[:, None] \
        * rng.random(n)[:, None]
    R = rotation(ang)
    t = np.exp(rng.uniform(np.log(0.01), np.log(20.0), size=n))[:, None] * rng.normal(size=(n, 3))
    return dict(W=W, H=H, fx=fx, fy=fy, cx=cx, cy=cy, fxi=fxi, fyi=fyi, cxi=cxi, cyi=cyi,
                u=u, v=v, z=z, R=R, t=t)


@pytest.mark.parametrize("off_centre", [False, True], ids=["centred", "off-centre"])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_fp32_position_error_within_the_bound(seed, off_centre):
    d = draw(seed, 200_000, off_centre)
    eps_z = 1e-6
    # exact lift (FP64) and the stored FP32 one
    X64 = np.stack([(d["u"] - d["cxi"]) / d["fxi"] * d["z"], (d["v"] - d["cyi"]) / d["fyi"] * d["z"], d["z"]], -1)
    X = f32(X64)
    w = f32(U * MARGIN * (5 * np.abs(X[:, 0]) + 4 * np.abs(X[:, 1]) + 2 * X[:, 2] + 2 * eps_z))
    # exact transform and projection
    Y64 = np.einsum("nij,nj->ni", d["R"], X64) + d["t"]
    front = Y64[:, 2] > 0.05
    # the kernel's FP32 steps
    r = f32(d["R"])
    tf = f32(d["t"])
    Y = np.empty_like(Y64)
    for k in range(3):
        Y[:, k] = fma32(r[:, k, 2], X[:, 2], fma32(r[:, k, 1], X[:, 1], fma32(r[:, k, 0], X[:, 0], tf[:, k])))
    Et = f32(4.0 * U * MARGIN * np.abs(tf).sum(axis=1))
    E = f32(w + Et)
    # every component of Y within E
    assert np.all(np.abs(Y - Y64)[front] <= E[front, None])
    # projection: rcp.approx carries up to 2u relative error; take it at its worst, either sign
    sgn = np.where(np.random.default_rng(seed + 7).random(len(E)) < 0.5, -1.0, 1.0)
    iz = f32(f32(1.0 / Y[:, 2]) * (1.0 + sgn * 2.0 * U))
    fxf, fyf, cxf, cyf = f32(d["fx"]), f32(d["fy"]), f32(d["cx"]), f32(d["cy"])
    up = fma32(fxf, f32(Y[:, 0] * iz), cxf)
    vp = fma32(fyf, f32(Y[:, 1] * iz), cyf)
    U64 = d["fx"] * Y64[:, 0] / Y64[:, 2] + d["cx"]
    V64 = d["fy"] * Y64[:, 1] / Y64[:, 2] + d["cy"]
    Kb, cb = bound_constants(d["fx"], d["fy"], d["cx"], d["cy"], d["W"], d["H"])
    tb = fma32(f32(E * iz), Kb, cb)
    near_image = (up >= -1) & (up <= d["W"]) & (vp >= -1) & (vp <= d["H"])
    sel = front & near_image & (tb <= 0.25)
    assert sel.sum() > 5_000  # enough samples land in the image to mean something
    err = np.maximum(np.abs(up - U64), np.abs(vp - V64))
    assert np.all(err[sel] <= tb[sel])
    # the bound is not loose by orders of magnitude: the worst sample uses a fair part of it
    assert (err[sel] / tb[sel]).max() > 0.05


def test_samples_far_outside_stay_outside():
    """A sample that FP32 puts s >= 1 outside the image with t <= 1/4 is outside in the exact
    evaluation too, however large its |xn| (the kernel drops it without the exact path)."""
    d = draw(11, 200_000, True)
    X64 = np.stack([(d["u"] - d["cxi"]) / d["fxi"] * d["z"], (d["v"] - d["cyi"]) / d["fyi"] * d["z"], d["z"]], -1)
    X = f32(X64)
    w = f32(U * MARGIN * (5 * np.abs(X[:, 0]) + 4 * np.abs(X[:, 1]) + 2 * X[:, 2] + 2e-6))
    Y64 = np.einsum("nij,nj->ni", d["R"], X64) + d["t"]
    r, tf = f32(d["R"]), f32(d["t"])
    Y = np.empty_like(Y64)
    for k in range(3):
        Y[:, k] = fma32(r[:, k, 2], X[:, 2], fma32(r[:, k, 1], X[:, 1], fma32(r[:, k, 0], X[:, 0], tf[:, k])))
    E = f32(w + f32(4.0 * U * MARGIN * np.abs(tf).sum(axis=1)))
    iz = f32(1.0 / Y[:, 2])
    up = fma32(f32(d["fx"]), f32(Y[:, 0] * iz), f32(d["cx"]))
    U64 = d["fx"] * Y64[:, 0] / Y64[:, 2] + d["cx"]
    Kb, cb = bound_constants(d["fx"], d["fy"], d["cx"], d["cy"], d["W"], d["H"])
    tb = fma32(f32(E * iz), Kb, cb)
    s_left, s_right = -up, up - (d["W"] - 1)
    out = (Y64[:, 2] > 0.05) & (tb <= 0.25) & ((s_left >= 1) | (s_right >= 1))
    assert out.sum() > 5_000
    exact_outside = (U64 < 0) | (U64 > d["W"] - 1)
    assert np.all(exact_outside[out])
