"""Stochastic viewgraph sub-sampling on the GPU (Algorithm 3, Appendix A.3: a fresh uniform
random subset of min(|E|, M) pairs every step) against the oracle.

The subset is integer work and is compared bit for bit: the device draws it from the step
counter with the same counter-based generator (SplitMix64 keys of (seed, step, pair)) that the
oracle implements independently.  The loss and gradient of a budgeted evaluation follow the
tolerances of the pose-only parity tests, on the oracle restricted to the drawn pairs."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import gpu_scene, oracle_maps_f32, scene_part
from tests.test_gpu_parity import check_against_oracle, oracle_of

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA GPU required", allow_module_level=True)

import paper_2607_00579_gb300 as epo  # noqa: E402

B = epo._binding
SEED = 0x5EED2607


@pytest.fixture(scope="module")
def ring8():
    sc = synth.make_scene(synth.RING8_128x96)
    return sc, oracle_maps_f32(sc)


def test_device_subsets_equal_oracle_subsets(ring8):
    sc, maps = ring8
    s = gpu_scene(sc, maps, pair_budget=20, subsample_seed=SEED)
    s.set_poses(sc.T_init)
    assert s.info().kernels_per_step == 4
    for step in range(6):
        s.step(1)  # step `step` draws its subset from the device step counter
        got = B.epo_get_pair_active(s.handle, sc.n_pairs)
        assert np.array_equal(got, oracle.subsample(SEED, step, sc.n_pairs, 20)), step


def test_budgeted_loss_and_gradient_match_oracle_on_the_drawn_pairs(ring8):
    sc, maps = ring8
    s = gpu_scene(sc, maps, pair_budget=20, subsample_seed=SEED)
    s.set_poses(sc.T_init)
    loss, grad = s.loss_and_grad()  # step counter 0
    ids = np.flatnonzero(oracle.subsample(SEED, 0, sc.n_pairs, 20))
    assert np.array_equal(np.flatnonzero(B.epo_get_pair_active(s.handle, sc.n_pairs)), ids)
    o = oracle.OracleScene(sc.W, sc.H, sc.K, sc.rec_off, sc.rec, [m.astype(np.float64) for m in maps],
                           sc.pairs[ids]).loss_grad(sc.T_init, lam=10.0)
    check_against_oracle(loss[0], grad, o, sc.pairs[ids], sc.T_init)


def test_budgeted_optimisation_tracks_oracle(ring8):
    sc, maps = ring8
    kw = dict(lr_rot=2e-3, lr_trans=5e-2)
    s = gpu_scene(sc, maps, pair_budget=20, subsample_seed=SEED, **kw)
    s.set_poses(sc.T_init)
    o = oracle_of(sc, maps)
    To, _, _, _ = o.optimize(sc.T_init, sc.fixed, 30, pair_budget=20, seed=SEED, **kw)
    step = 0
    for c in (10, 20, 30):
        s.step(c - step)
        step = c
    Tg = s.get_poses()
    # same subsets every step; the poses agree as closely as the pose-only 50-step test
    from tests.helpers import rot_err_deg, trans_err
    assert rot_err_deg(Tg, To).max() <= 0.01
    assert trans_err(Tg, To, sc.scale).max() <= 1e-4
    assert rot_err_deg(Tg, sc.T_gt).mean() < rot_err_deg(sc.T_init, sc.T_gt).mean()


def test_large_scene_subset_and_batched_scenes():
    spec = synth.RING500_518x518
    sc = synth.make_scene(spec)
    maps = oracle_maps_f32(sc)
    s = gpu_scene(sc, maps, pair_budget=1024, subsample_seed=SEED)
    s.set_poses(sc.T_init)
    s.loss_and_grad()
    assert np.array_equal(B.epo_get_pair_active(s.handle, sc.n_pairs), oracle.subsample(SEED, 0, sc.n_pairs, 1024))
    # a batch: every scene draws from its own pairs (indices within the scene)
    specs = synth.batch64_uneven_specs(n_scenes=3)
    for sp in specs:
        sp.width, sp.height, sp.n_views = 160, 120, min(sp.n_views, 12)
    scenes = [synth.make_scene(sp) for sp in specs]
    b = epo.Scene([scene_part(x, oracle_maps_f32(x)) for x in scenes],
                  options=epo.default_options(pair_budget=30, subsample_seed=SEED))
    b.set_poses(np.concatenate([x.T_init for x in scenes]))
    b.loss_and_grad()
    act = B.epo_get_pair_active(b.handle, sum(x.n_pairs for x in scenes))
    off = 0
    for x in scenes:
        assert np.array_equal(act[off:off + x.n_pairs], oracle.subsample(SEED, 0, x.n_pairs, 30))
        off += x.n_pairs


def test_subset_hook_refused_with_a_budget(ring8):
    sc, maps = ring8
    s = gpu_scene(sc, maps, pair_budget=20)
    with pytest.raises(epo.EpoError):
        s.set_pair_subset([1, 2, 3])
