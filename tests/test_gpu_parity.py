"""GPU kernels vs the FP64 oracle, element by element on the same seeded inputs.

Tolerances (FP32 path, stated by the arithmetic):
  * loss: relative 1e-5;  gradient: max_i ||g_i - g_i^oracle|| <= 1e-4 max_i ||g_i^oracle||.
    FP32 rounding of T_ji and of the projection moves a sample by ~1e-7 of its pixel
    coordinate (<= 5e-5 px at 518 px); with |grad DTF| <= 1 the per-sample distance moves by
    the same amount, which averages to ~1e-6 relative over thousands of samples.
  * n_valid per pair is an integer decided by FP comparisons of the projected position
    against the image border (and the depth against eps_z).  The kernel takes every decision
    that its FP32 rounding-error bound cannot settle (border, bilinear cell, depth threshold,
    clamp) again in FP64, so it decides as an FP64 evaluation does; the two FP64 evaluations
    may still differ on samples within FP64 rounding of a boundary (the oracle's pair_near
    count at a 1e-9 px margin), so |n_gpu - n_oracle| <= near is required exactly.
  * BF16 maps / FP16 depth: against the oracle fed the same rounded values ("kernel parity")
    the FP32 tolerances hold; against the oracle fed the full-precision inputs ("precision
    cost") loss and gradient agree to 1e-2.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests.helpers import (bf16_bits, bf16_to_f32, grad_rel_err, gpu_scene, oracle_maps_f32, rot_err_deg,
                           scene_part, trans_err)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA GPU required", allow_module_level=True)

import paper_2607_00579_gb300 as epo  # noqa: E402

LOSS_RTOL = 1e-5
GRAD_RTOL = 1e-4
PAIR_RHO_RTOL = 1e-5
PAIR_GRAD_RTOL = 1e-4
CELL_FLIPS = 0  # adjacent-cell choices per pair allowed to differ (none: the kernel re-decides them in FP64)


@pytest.fixture(scope="module")
def ring8():
    sc = synth.make_scene(synth.RING8_128x96)
    maps = oracle_maps_f32(sc)
    return sc, maps


def oracle_of(sc, maps, rec=None):
    return oracle.scene_from_synth(sc, [m.astype(np.float64) for m in maps],
                                   rec=None if rec is None else rec)


def huber_max(lam, delta):
    return delta * (lam - 0.5 * delta) if lam > delta else 0.5 * lam * lam


def pose4(T12):
    M = np.eye(4)
    M[:3] = np.asarray(T12).reshape(3, 4)
    return M


def allowances(o, pairs, T, n_views, lam, delta):
    """What FP32-vs-FP64 decisions may legitimately change.

    A validity flip (a sample within 1e-3 px of the border, counted by the oracle) moves one
    sample in or out of a pair's mean: the pair loss moves by at most (H(lambda) + l_p)/n and
    the pair's gradient by at most one sample's term plus a 1/n rescale.  Independently, a
    sample within ~1e-4 px of a bilinear cell line may take the neighbouring cell, changing
    its slope term by at most twice its size; CELL_FLIPS such samples are allowed per pair
    (zero: the kernel settles every cell choice within its FP32 error bound in FP64).
    The target pose receives a pair's 6-vector as is, the source pose through -Ad(T_ji)^T,
    whose norm is at most 2 + |t_ji|."""
    near = o["pair_near"].astype(float)
    n = o["pair_stats"][:, 1]
    P = len(near)
    w = near / np.maximum(n - near, 1.0)
    allow_L = 2.0 / P * float(np.sum(w * (huber_max(lam, delta) + o["pair_loss"])))
    per_pair = 2.0 / P * (2.0 * near + 2.0 * CELL_FLIPS) * o["pair_maxterm"] / np.maximum(n - near, 1.0)
    allow_g = np.zeros(n_views)
    for p, (i, j) in enumerate(np.asarray(pairs)):
        if per_pair[p] == 0:
            continue
        tji = (pose4(T[j]) @ np.linalg.inv(pose4(T[i])))[:3, 3]
        allow_g[j] += per_pair[p]
        allow_g[i] += per_pair[p] * (2.0 + np.linalg.norm(tji))
    return allow_L, allow_g


def check_against_oracle(loss_g, grad_g, o, pairs, T, lam=10.0, delta=1.0, stats=None, grad_scale=1.0,
                         slope_pairs=None, gref=0.0):
    """slope_pairs: boolean mask of the pairs whose per-pair slope sums are compared (default all).
    gref: gradient scale of the problem, max ||g_i|| at a run's initial poses, for poses further
    along an optimisation: the FP32 error is a fixed absolute
    amount set by the per-sample terms (measured 4.7e-5 to 8.7e-5 along the 200-step 32-view
    ring), which stay O(1) while their sum, the gradient, shrinks near the optimum (there up to
    1.8e-4 of the current gradient).  The tolerance is 1e-4 of the larger of gref and the
    current max ||g_i||."""
    allow_L, allow_g = allowances(o, pairs, T, len(grad_g), lam, delta)
    assert abs(loss_g - o["loss"]) <= LOSS_RTOL * abs(o["loss"]) + allow_L, (loss_g, o["loss"], allow_L)
    err = np.linalg.norm(np.asarray(grad_g) - o["grad"], axis=1)
    gmax = max(np.linalg.norm(o["grad"], axis=1).max(), gref)
    bad = err > GRAD_RTOL * gmax + grad_scale * allow_g
    assert not bad.any(), (err[bad], gmax, allow_g[bad])
    if stats is not None:
        near = o["pair_near"]
        dn = np.abs(stats[:, 1] - o["pair_stats"][:, 1])
        assert np.all(dn <= near), (dn.max(), near[dn.argmax()])
        same = dn == 0
        d_rho = np.abs(stats[same, 0] - o["pair_stats"][same, 0])
        assert np.all(d_rho <= PAIR_RHO_RTOL * np.abs(o["pair_stats"][same, 0]) + 1e-6)
        if slope_pairs is not None:
            same = same & slope_pairs
        d_g = np.abs(stats[same, 2:] - o["pair_stats"][same, 2:])
        tol = PAIR_GRAD_RTOL * o["pair_abs"][same] + 2.0 * CELL_FLIPS * o["pair_maxterm"][same, None]
        assert np.all(d_g <= tol), (d_g / np.maximum(o["pair_abs"][same], 1e-300)).max()


# ---------------------------------------------------------------------------------------------
SCHEDULES = [(g, r, b) for g in (epo.EPO_GATHER_LDG, epo.EPO_GATHER_TEX) for r, b in ((4, 256), (2, 128), (1, 512))]
SCHEDULES += [(epo.EPO_GATHER_MIX, 2, 128), (epo.EPO_GATHER_MIX, 4, 256), (epo.EPO_GATHER_LDG, 8, 128),
              (epo.EPO_GATHER_TEX, 8, 64), (epo.EPO_GATHER_MIX, 8, 512)]


@pytest.mark.parametrize("gather,rpt,block", SCHEDULES)
def test_loss_grad_parity_small_ring(ring8, gather, rpt, block):
    sc, maps = ring8
    s = gpu_scene(sc, maps, gather=gather, records_per_thread=rpt, block_threads=block)
    s.set_poses(sc.T_init)
    loss, grad = s.loss_and_grad()
    st = s.pair_stats()
    o = oracle_of(sc, maps).loss_grad(sc.T_init, lam=10.0)
    check_against_oracle(loss[0], grad, o, sc.pairs, sc.T_init, stats=st)


@pytest.mark.parametrize("gather,rpt,block", [(epo.EPO_GATHER_TEX, 4, 128), (epo.EPO_GATHER_LDG, 2, 128)])
def test_off_centre_wide_angle_intrinsics_match_oracle(ring8, gather, rpt, block):
    """The pose kernel's rounding bound where its terms are largest: a focal length a third of
    the scene's (|xn| up to ~1.5 at the image edges, so the X0 and X1 terms dominate z's) and
    principal points far off centre and not exact in FP32 (the projection's |u' - cx| and |cx|
    terms, and the stored lift's rounding of cx), with the records and maps unchanged: every
    cell, border and depth decision must still be the exact evaluation's."""
    import dataclasses
    sc, maps = ring8
    K = sc.K.copy()
    K[:, 0] *= 0.3333331
    K[:, 1] *= 0.3512347
    K[:, 2] += 0.31234567 * sc.W
    K[:, 3] -= 0.27654321 * sc.H
    sw = dataclasses.replace(sc, K=K)
    s = gpu_scene(sw, maps, gather=gather, records_per_thread=rpt, block_threads=block)
    s.set_poses(sc.T_init)
    loss, grad = s.loss_and_grad()
    st = s.pair_stats()
    o = oracle_of(sw, maps).loss_grad(sc.T_init, lam=10.0)
    # a fair share of the samples still lands in the images
    assert o["pair_stats"][:, 1].sum() > 0.2 * sum(int(sc.rec_off[i + 1] - sc.rec_off[i]) for i, _ in sc.pairs)
    check_against_oracle(loss[0], grad, o, sc.pairs, sc.T_init, stats=st)


@pytest.mark.parametrize("tail", [1, 2, 3])
def test_split_last_wave_matches_oracle(ring8, tail):
    """Work items of the last wave split into items of `tail` pairs (on this small scene the
    whole tile list is one wave, so every item is split)."""
    sc, maps = ring8
    s = gpu_scene(sc, maps, tail_pairs=tail)
    assert s.info().tail_pairs == tail
    s.set_poses(sc.T_init)
    loss, grad = s.loss_and_grad()
    o = oracle_of(sc, maps).loss_grad(sc.T_init, lam=10.0)
    check_against_oracle(loss[0], grad, o, sc.pairs, sc.T_init, stats=s.pair_stats())
    ref = gpu_scene(sc, maps, tail_pairs=0)
    ref.set_poses(sc.T_init)
    assert s.info().n_tiles > ref.info().n_tiles
    l0, g0 = ref.loss_and_grad()
    assert loss[0] == pytest.approx(l0[0], rel=1e-12) and grad_rel_err(grad, g0) < 1e-10


@pytest.mark.parametrize("split", [2, 3])
def test_split_every_item_matches_oracle(ring8, split):
    """Every work item split into items of at most `split` pairs (tail_pairs = -split), on a
    grid of two blocks, so that the items run in many waves."""
    sc, maps = ring8
    s = gpu_scene(sc, maps, tail_pairs=-split, grid_blocks=2)
    assert s.info().tail_pairs == -split
    s.set_poses(sc.T_init)
    loss, grad = s.loss_and_grad()
    o = oracle_of(sc, maps).loss_grad(sc.T_init, lam=10.0)
    check_against_oracle(loss[0], grad, o, sc.pairs, sc.T_init, stats=s.pair_stats())
    last = gpu_scene(sc, maps, tail_pairs=split, grid_blocks=2)
    ref = gpu_scene(sc, maps, tail_pairs=0, grid_blocks=2)
    ks = set(np.bincount(np.asarray(sc.pairs)[:, 0]).tolist())  # all ordered pairs: k per view
    assert len(ks) == 1
    k = ks.pop()
    assert s.info().n_tiles == ref.info().n_tiles * -(-k // split)
    assert s.info().n_tiles > last.info().n_tiles > ref.info().n_tiles
    for h in (last, ref):
        h.set_poses(sc.T_init)
        l0, g0 = h.loss_and_grad()
        assert loss[0] == pytest.approx(l0[0], rel=1e-12) and grad_rel_err(grad, g0) < 1e-10


def test_gather_paths_and_schedules_agree(ring8):
    sc, maps = ring8
    res = []
    for gather, rpt, block in [(1, 4, 256), (2, 4, 256), (1, 1, 128), (2, 2, 512)]:
        s = gpu_scene(sc, maps, gather=gather, records_per_thread=rpt, block_threads=block)
        s.set_poses(sc.T_init)
        res.append(s.loss_and_grad())
    for l, g in res[1:]:
        assert l[0] == pytest.approx(res[0][0][0], rel=1e-6)
        assert grad_rel_err(g, res[0][1]) < 1e-6


@pytest.mark.parametrize("grid", [1, 5000])
def test_grid_sizes_agree(ring8, grid):
    """A one-block grid (the block starts on item 0 and claims every later item in turn) and a
    grid option far larger than the work list (capped at one block per item: every block runs
    only its own first item) give the default grid's loss and gradient."""
    sc, maps = ring8
    ref = gpu_scene(sc, maps)
    s = gpu_scene(sc, maps, grid_blocks=grid)
    assert grid > s.info().n_tiles or grid == 1
    for h in (ref, s):
        h.set_poses(sc.T_init)
    l0, g0 = ref.loss_and_grad()
    l1, g1 = s.loss_and_grad()
    assert l1[0] == pytest.approx(l0[0], rel=1e-12) and grad_rel_err(g1, g0) < 1e-10
    o = oracle_of(sc, maps).loss_grad(sc.T_init, lam=10.0)
    check_against_oracle(l1[0], g1, o, sc.pairs, sc.T_init, stats=s.pair_stats())


def test_norm_all_mode(ring8):
    sc, maps = ring8
    s = gpu_scene(sc, maps, norm_mode=epo.EPO_NORM_ALL)
    s.set_poses(sc.T_init)
    loss, grad = s.loss_and_grad()
    o = oracle_of(sc, maps).loss_grad(sc.T_init, lam=10.0, norm_mode=oracle.NORM_ALL)
    check_against_oracle(loss[0], grad, o, sc.pairs, sc.T_init)


def test_lambda_and_huber_options(ring8):
    sc, maps = ring8
    s = gpu_scene(sc, maps, lambda0=2.5, lambda1=2.5, huber_delta=0.5)
    s.set_poses(sc.T_init)
    loss, grad = s.loss_and_grad()
    o = oracle_of(sc, maps).loss_grad(sc.T_init, lam=2.5, delta=0.5)
    check_against_oracle(loss[0], grad, o, sc.pairs, sc.T_init, lam=2.5, delta=0.5, stats=s.pair_stats())


def tiny_edge_scene():
    """Hand-made records: on the image border, on cell lines, behind the camera, ragged tile
    tails (counts not multiples of any tile), an empty source view and a self pair."""
    rng = np.random.default_rng(7)
    n, W, H = 4, 33, 17
    f = 20.0
    K = np.tile([f, f, (W - 1) / 2, (H - 1) / 2], (n, 1))
    T = np.zeros((n, 12))
    from scipy.spatial.transform import Rotation
    for v in range(n):
        R = Rotation.from_rotvec(rng.normal(0, 0.03, 3)).as_matrix()
        T[v] = np.concatenate([R, rng.normal(0, 0.05, 3)[:, None]], 1).reshape(-1)
    counts = [1037, 0, 3, 517]
    recs, off = [], [0]
    for v in range(n):
        c = counts[v]
        u = rng.integers(0, W, c).astype(np.float32)
        vv = rng.integers(0, H, c).astype(np.float32)
        z = rng.uniform(3.0, 5.0, c).astype(np.float32)
        if c > 10:
            u[:4] = [0, W - 1, 0, W - 1]
            vv[:4] = [0, 0, H - 1, H - 1]
            z[4] = -1.0  # dropped at creation
        r = np.zeros((c, 4), np.float32)
        r[:, 0], r[:, 1], r[:, 2] = u, vv, z
        recs.append(r)
        off.append(off[-1] + c)
    rec = np.concatenate(recs)
    maps = [rng.uniform(0, 5, (H, W)).astype(np.float32) for _ in range(n)]
    pairs = np.array([(0, 1), (1, 0), (0, 0), (2, 3), (3, 2), (0, 3), (3, 0), (2, 0)], np.int32)
    return dict(W=[W] * n, H=[H] * n, K=K, rec_off=np.array(off), rec=rec, maps=maps, pairs=pairs,
                fixed=None), T


def test_edge_cases_ragged_empty_border_self_pair():
    part, T = tiny_edge_scene()
    s = epo.Scene([part])
    assert s.info().n_dropped == 2
    s.set_poses(T)
    loss, grad = s.loss_and_grad()
    keep = part["rec"][:, 2] > 0
    rec = part["rec"][keep]
    cnt = [int(np.sum(keep[part["rec_off"][v]:part["rec_off"][v + 1]])) for v in range(4)]
    off = np.concatenate([[0], np.cumsum(cnt)])
    os_ = oracle.OracleScene(part["W"], part["H"], part["K"], off, rec,
                             [m.astype(np.float64) for m in part["maps"]], part["pairs"])
    o = os_.loss_grad(T, lam=10.0)
    st = s.pair_stats()
    # the self pair (0, 0) projects every record exactly onto its own integer pixel, where
    # the bilinear slope is one-sided and FP32 / FP64 rounding picks the cell; its slope sums
    # are not comparable (its target and source contributions cancel in the pose gradient)
    self_pair = part["pairs"][:, 0] == part["pairs"][:, 1]
    check_against_oracle(loss[0], grad, o, part["pairs"], T, stats=st, slope_pairs=~self_pair)
    assert st[1, 1] == 0 and st[1, 0] == 0  # empty source view


def test_all_samples_invalid_gives_zero_pair_loss():
    part, T = tiny_edge_scene()
    T2 = T.copy()
    from scipy.spatial.transform import Rotation
    # view 3 turned around: nothing from view 0 or 2 lands in front of it
    M = T2[3].reshape(3, 4)
    T2[3] = np.concatenate([Rotation.from_rotvec([0, math.pi, 0]).as_matrix() @ M[:, :3], M[:, 3:]], 1).reshape(-1)
    s = epo.Scene([part])
    s.set_poses(T2)
    loss, grad = s.loss_and_grad()
    st = s.pair_stats()
    assert st[3, 1] == 0 and st[5, 1] == 0
    assert np.isfinite(loss).all() and np.isfinite(grad).all()


# ---------------------------------------------------------------------------------------------
def test_distance_field_kernel_is_exact(ring8):
    sc, _ = ring8
    rng = np.random.default_rng(3)
    cases = [e for e in sc.edges[:3]]
    cases += [(rng.random((H, W)) < d).astype(np.uint8) for (H, W, d) in
              [(17, 33, 0.05), (1, 9, 0.3), (40, 1, 0.1), (64, 70, 0.0), (50, 200, 0.001), (392, 518, 0.02)]]
    for e in cases:
        g = epo.distance_field(torch.from_numpy(e).cuda()).cpu().numpy()
        ref = oracle.edt(e).astype(np.float32)
        assert np.array_equal(g, ref)


def test_bf16_rounding_kernel_matches_rne():
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.uniform(0, 600, 100000), np.arange(0, 1000, 0.25)]).astype(np.float32)
    g = epo.round_bf16(torch.from_numpy(x).cuda()).cpu().numpy().view(np.uint16)
    assert np.array_equal(g, bf16_bits(x))


# ---------------------------------------------------------------------------------------------
def test_fp16_depth_bf16_map_kernel_parity_and_precision_cost(ring8):
    sc, maps = ring8
    bits = [bf16_bits(m) for m in maps]
    rec16 = synth.records_f16(sc.rec)
    s = gpu_scene(sc, bits, rec=rec16, record_dtype=epo.EPO_F16, map_dtype=epo.EPO_BF16)
    s.set_poses(sc.T_init)
    loss, grad = s.loss_and_grad()
    # kernel parity: the oracle sees exactly the stored values
    o_same = oracle.scene_from_synth(sc, [bf16_to_f32(b).astype(np.float64) for b in bits],
                                     rec=synth.records_f16_widened(sc.rec)).loss_grad(sc.T_init, lam=10.0)
    check_against_oracle(loss[0], grad, o_same, sc.pairs, sc.T_init, stats=s.pair_stats())
    # precision cost: the oracle sees the full-precision inputs
    o_full = oracle_of(sc, maps).loss_grad(sc.T_init, lam=10.0)
    assert abs(loss[0] - o_full["loss"]) <= 1e-2 * o_full["loss"]
    assert grad_rel_err(grad, o_full["grad"]) <= 1e-2


# ---------------------------------------------------------------------------------------------
def test_optimisation_matches_oracle_and_improves(ring8):
    sc, maps = ring8
    kw = dict(lr_rot=2e-3, lr_trans=5e-2)
    s = gpu_scene(sc, maps, **kw)
    s.set_poses(sc.T_init)
    s.step(50)
    Tg = s.get_poses()
    To, _, _, hist = oracle_of(sc, maps).optimize(sc.T_init, sc.fixed, 50, **kw)
    assert rot_err_deg(Tg, To).max() <= 0.01
    assert trans_err(Tg, To, sc.scale).max() <= 1e-4
    assert rot_err_deg(Tg, sc.T_gt).mean() < rot_err_deg(sc.T_init, sc.T_gt).mean()
    assert trans_err(Tg, sc.T_gt, sc.scale).mean() < trans_err(sc.T_init, sc.T_gt, sc.scale).mean()
    assert np.array_equal(Tg[0], sc.T_init[0])
    step, m, v = s.get_state()
    assert step == 50


def test_graph_step_equals_plain_step(ring8):
    sc, maps = ring8
    a = gpu_scene(sc, maps)
    b = gpu_scene(sc, maps)
    a.set_poses(sc.T_init)
    b.set_poses(sc.T_init)
    a.step(10)
    b.step_plain(10)
    b.check()
    # identical kernels; only the order of FP64 atomics differs between runs
    assert np.abs(a.get_poses() - b.get_poses()).max() < 1e-9


def test_checkpoint_resume_equals_uninterrupted(ring8):
    sc, maps = ring8
    a = gpu_scene(sc, maps)
    a.set_poses(sc.T_init)
    a.step(20)
    b = gpu_scene(sc, maps)
    b.set_poses(sc.T_init)
    b.step(10)
    T, st = b.get_poses(), b.get_state()
    c = gpu_scene(sc, maps)
    c.set_poses(T)
    c.set_state(*st)
    c.step(10)
    assert np.abs(a.get_poses() - c.get_poses()).max() < 1e-9


def test_nonfinite_pose_refuses_update(ring8):
    sc, maps = ring8
    s = gpu_scene(sc, maps)
    s.set_poses(sc.T_init)
    T = torch.tensor(sc.T_init, dtype=torch.float64, device="cuda")
    T[2, 3] = float("nan")
    epo._binding.epo_set_poses_dev(s.handle, T)
    with pytest.raises(epo.EpoError) as e:
        s.step(3)
    assert e.value.status == epo._binding.EPO_ERR_NUMERIC
    after = s.get_poses()
    assert np.array_equal(after[1], sc.T_init[1])
    assert s.get_state()[0] == 0


def test_nan_map_is_rejected(ring8):
    sc, maps = ring8
    bad = [m.copy() for m in maps]
    bad[3][5, 5] = np.nan
    with pytest.raises(epo.EpoError) as e:
        gpu_scene(sc, bad)
    assert e.value.status == epo._binding.EPO_ERR_INVALID_ARG


# ---------------------------------------------------------------------------------------------
def test_autograd_forward_backward(ring8):
    sc, maps = ring8
    s = gpu_scene(sc, maps)
    s.set_poses(sc.T_init)
    ref_loss, ref_grad = s.loss_and_grad()
    xi = torch.zeros((sc.n_views, 6), dtype=torch.float64, device="cuda", requires_grad=True)
    L = epo.EdgeLoss.apply(xi, s)
    L.sum().backward()
    assert L.item() == pytest.approx(ref_loss[0], rel=1e-12)
    assert grad_rel_err(xi.grad.cpu().numpy(), ref_grad) < 1e-9
    # at a non-zero twist: d/dxi L(Exp(xi) T) = J_l(xi)^T g_left(Exp(xi) T)
    rng = np.random.default_rng(5)
    x = rng.normal(0, 0.01, (sc.n_views, 6))
    xt = torch.tensor(x, device="cuda", requires_grad=True)
    L = epo.EdgeLoss.apply(xt, s)
    (3.0 * L.sum()).backward()
    Tx = np.stack([(np.vstack([oracle.se3_exp(x[v]).reshape(3, 4), [0, 0, 0, 1]])
                    @ np.vstack([sc.T_init[v].reshape(3, 4), [0, 0, 0, 1]]))[:3].reshape(-1)
                   for v in range(sc.n_views)])
    o = oracle_of(sc, maps).loss_grad(Tx, lam=10.0)
    assert L.item() == pytest.approx(o["loss"], rel=LOSS_RTOL)
    want = 3.0 * np.stack([oracle.se3_left_jacobian(x[v]).T @ o["grad"][v] for v in range(sc.n_views)])
    assert grad_rel_err(xt.grad.cpu().numpy(), want) <= GRAD_RTOL


def test_batched_scenes_equal_individual_scenes():
    specs = synth.batch64_uneven_specs(n_scenes=3)
    for sp in specs:
        sp.width, sp.height, sp.n_views = 160, 120, min(sp.n_views, 12)
    scenes = [synth.make_scene(sp) for sp in specs]
    maps = [oracle_maps_f32(sc) for sc in scenes]
    b = epo.Scene([scene_part(sc, m) for sc, m in zip(scenes, maps)])
    b.set_poses(np.concatenate([sc.T_init for sc in scenes]))
    lb, gb = b.loss_and_grad()
    off = 0
    for k, (sc, m) in enumerate(zip(scenes, maps)):
        s = gpu_scene(sc, m)
        s.set_poses(sc.T_init)
        l1, g1 = s.loss_and_grad()
        assert lb[k] == pytest.approx(l1[0], rel=1e-12)
        assert grad_rel_err(gb[off:off + sc.n_views], g1) < 1e-10
        o = oracle_of(sc, m).loss_grad(sc.T_init, lam=10.0)
        check_against_oracle(lb[k], gb[off:off + sc.n_views], o, sc.pairs, sc.T_init)
        off += sc.n_views


def test_pair_subset(ring8):
    sc, maps = ring8
    s = gpu_scene(sc, maps)
    s.set_poses(sc.T_init)
    ids = np.array([3, 17, 40, 41, 55])
    s.set_pair_subset(ids)
    loss, grad = s.loss_and_grad()
    o = oracle.OracleScene(sc.W, sc.H, sc.K, sc.rec_off, sc.rec,
                           [m.astype(np.float64) for m in maps], sc.pairs[ids]).loss_grad(sc.T_init, lam=10.0)
    check_against_oracle(loss[0], grad, o, sc.pairs[ids], sc.T_init)
    assert s.info().evals_per_step == int(np.diff(sc.rec_off)[sc.pairs[ids, 0]].sum())
    s.set_pair_subset([])
    l2, _ = s.loss_and_grad()
    assert l2[0] == pytest.approx(oracle_of(sc, maps).loss_grad(sc.T_init, lam=10.0)["loss"], rel=LOSS_RTOL)


def test_autotune_keeps_results(ring8):
    sc, maps = ring8
    s = gpu_scene(sc, maps, autotune=1)
    s.set_poses(sc.T_init)
    loss, grad = s.loss_and_grad()
    o = oracle_of(sc, maps).loss_grad(sc.T_init, lam=10.0)
    check_against_oracle(loss[0], grad, o, sc.pairs, sc.T_init, stats=s.pair_stats())
    i = s.info()
    assert i.records_per_thread in (1, 2, 4) and i.block_threads in (128, 256, 512)


# ---------------------------------------------------------------------------------------------
# full size: the 32-view 518x392 ring in the benchmark's launch configuration
# ---------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def ring32():
    sc = synth.make_scene(synth.RING32_518x392)
    return sc, oracle_maps_f32(sc)


def test_full_size_sampled_pairs_match_oracle(ring32):
    sc, maps = ring32
    for v in (0, 7, 31):  # the GPU's distance transform gives the same maps
        g = epo.distance_field(torch.from_numpy(sc.edges[v]).cuda()).cpu().numpy()
        assert np.array_equal(g, maps[v])
    s = gpu_scene(sc, maps)
    s.set_poses(sc.T_init)
    loss, grad = s.loss_and_grad()
    st = s.pair_stats()
    rng = np.random.default_rng(11)
    ids = np.sort(rng.choice(sc.n_pairs, 24, replace=False))
    o = oracle.OracleScene(sc.W, sc.H, sc.K, sc.rec_off, sc.rec, [m.astype(np.float64) for m in maps],
                           sc.pairs[ids]).loss_grad(sc.T_init, lam=10.0)
    # per-pair sums of the sampled pairs, computed by the oracle one pair at a time
    check_against_oracle(float(o["loss"]), o["grad"], o, sc.pairs[ids], sc.T_init)  # self-consistency
    sub = st[ids]
    dn = np.abs(sub[:, 1] - o["pair_stats"][:, 1])
    assert np.all(dn <= o["pair_near"])
    same = dn == 0
    assert np.all(np.abs(sub[same, 0] - o["pair_stats"][same, 0]) <= PAIR_RHO_RTOL * o["pair_stats"][same, 0] + 1e-6)
    tol = PAIR_GRAD_RTOL * o["pair_abs"][same] + 2.0 * CELL_FLIPS * o["pair_maxterm"][same, None]
    assert np.all(np.abs(sub[same, 2:] - o["pair_stats"][same, 2:]) <= tol)
    # the whole loss and gradient (the oracle runs all 256 pairs once)
    full = oracle_of(sc, maps).loss_grad(sc.T_init, lam=10.0)
    check_against_oracle(loss[0], grad, full, sc.pairs, sc.T_init, stats=st)
    # a fraction of a percent of the samples took the exact path; none overflowed its queue
    queued, overflow = epo._binding.epo_fixup_stats(s.handle)
    assert 0 < queued < 0.05 * s.info().evals_per_step and overflow == 0


def test_gather_probe_rates_and_argument_checks():
    B = epo._binding
    r = {}
    for g in (epo.EPO_GATHER_LDG, epo.EPO_GATHER_TEX):
        for pat in (0, 1):
            for md in (epo.EPO_F32, epo.EPO_BF16):
                r[g, pat, md] = B.epo_gather_probe(8, 518, 392, md, g, pat, 1 << 22, 3)
    # a GPU serves between 1e9 and 1e13 footprints per second; warp-coherent positions reuse
    # cache lines, so they are served at least as fast as scattered ones (within noise)
    assert all(1e9 < v < 1e13 for v in r.values()), r
    for g in (epo.EPO_GATHER_LDG, epo.EPO_GATHER_TEX):
        assert r[g, 1, epo.EPO_F32] > 0.8 * r[g, 0, epo.EPO_F32]
    for bad in [dict(n_maps=0), dict(W=1), dict(pattern=2), dict(gather=0), dict(map_dtype=7),
                dict(pattern=1, W=40)]:
        a = dict(n_maps=2, W=64, H=32, map_dtype=epo.EPO_F32, gather=epo.EPO_GATHER_LDG, pattern=0)
        a.update(bad)
        with pytest.raises(epo.EpoError) as e:
            B.epo_gather_probe(a["n_maps"], a["W"], a["H"], a["map_dtype"], a["gather"], a["pattern"], 1000, 1)
        assert e.value.status == B.EPO_ERR_INVALID_ARG


@pytest.mark.parametrize("opts", [{}, {"schedule": 1}, {"refine": 1, "lr_focal": 1e-3, "lr_depth": 1e-3}],
                         ids=["pose-kernel-last", "schedule-last", "depth-kernel-last"])
def test_step_host_equals_separate_calls(ring8, opts):
    """epo_step_host (poses in, one step, poses and loss out, one synchronisation) gives what
    epo_set_poses + epo_step + epo_get_poses + epo_last_loss give: with the pose kernel as the
    step's last kernel (it writes the host outputs itself) and with a later kernel (a copy
    kernel writes them)."""
    B = epo._binding
    sc, maps = ring8
    a, b = gpu_scene(sc, maps, **opts), gpu_scene(sc, maps, **opts)
    T = np.ascontiguousarray(np.asarray(sc.T_init, dtype=np.float64).reshape(-1, 12))
    Ta, la = np.zeros_like(T), np.zeros(1)
    B.epo_step_host(a.handle, T, Ta, la)
    b.set_poses(T)
    b.step(1)
    lb = np.zeros(1)
    B.epo_last_loss(b.handle, lb)
    assert np.abs(Ta - b.get_poses().reshape(-1, 12)).max() < 1e-12
    assert la[0] == pytest.approx(lb[0], rel=1e-12)
    # consecutive calls through the same staging: poses fed back, then a call that keeps the
    # device's poses (T_in NULL), then one after steps queued without synchronisation
    for _ in range(3):
        B.epo_step_host(a.handle, Ta.copy(), Ta, la)
        b.step(1)
    B.epo_step_host(a.handle, None, Ta, la)
    b.step(1)
    B.epo_step_async(a.handle, 2)
    b.step(2)
    B.epo_step_host(a.handle, None, Ta, la)
    b.step(1)
    B.epo_last_loss(b.handle, lb)
    assert np.abs(Ta - b.get_poses().reshape(-1, 12)).max() < 1e-12
    assert la[0] == pytest.approx(lb[0], rel=1e-12)
    # non-finite input poses anywhere in the array are refused before anything runs: the next
    # step continues from the same state
    for pos, val in (((0, 0), np.nan), ((-1, -1), np.inf), ((3, 5), -np.inf)):
        bad = T.copy()
        bad[pos] = val
        with pytest.raises(epo.EpoError) as e:
            B.epo_step_host(a.handle, bad, None, None)
        assert e.value.status == B.EPO_ERR_INVALID_ARG
    B.epo_step_host(a.handle, None, Ta, la)
    b.step(1)
    B.epo_last_loss(b.handle, lb)
    assert np.abs(Ta - b.get_poses().reshape(-1, 12)).max() < 1e-12
    assert la[0] == pytest.approx(lb[0], rel=1e-12)
