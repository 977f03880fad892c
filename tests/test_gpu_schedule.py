"""The optimisation schedule on the GPU (Section 3, Optimization Schedule) against the oracle:
theta_95 of every step, computed on the device from the poses before and after the step,
equals the oracle's theta_95 of the same two pose sets; the device's dual-phase decisions
equal the oracle's rule fed the same theta_95 sequence; a converged scene stops moving."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import gpu_scene, oracle_maps_f32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA GPU required", allow_module_level=True)

import paper_2607_00579_gb300 as epo  # noqa: E402

B = epo._binding


@pytest.fixture(scope="module")
def ring8():
    sc = synth.make_scene(synth.RING8_128x96)
    return sc, oracle_maps_f32(sc)


def run_schedule(sc, maps, n, **cfg):
    """n single steps; returns theta_95 (device), phases (device), the oracle's theta_95 of the
    same poses, and whether the poses stayed fixed after convergence."""
    s = gpu_scene(sc, maps, schedule=1, lr_rot=1e-3, lr_trans=1e-2, **cfg)
    s.set_poses(sc.T_init)
    th_dev, phases, th_orc, frozen = [], [], [], True
    for _ in range(n):
        T0 = s.get_poses()
        phase_before = int(B.epo_get_schedule(s.handle, 1)[1][0])
        s.step(1)
        T1 = s.get_poses()
        th, ph, sw, st = B.epo_get_schedule(s.handle, 1)
        if phase_before == 3:
            frozen &= bool(np.array_equal(T0, T1))
            continue
        th_dev.append(th[0])
        phases.append(int(ph[0]))
        th_orc.append(oracle.theta95(T0, T1))
    return s, np.array(th_dev), phases, np.array(th_orc), frozen


def test_theta95_and_phase_changes_at_known_steps(ring8):
    sc, maps = ring8
    # every step's theta_95 is below 10 degrees: phase 2 after 3 steps, converged after 3 more
    cfg = dict(sched_eps1=10.0, sched_w1=3, sched_eps2=10.0, sched_w2=3)
    s, th, phases, th_o, frozen = run_schedule(sc, maps, 9, **cfg)
    assert np.allclose(th, th_o, rtol=1e-9, atol=1e-9)
    assert phases == [1, 1, 2, 2, 2, 3] and frozen
    _, ph, sw, st = B.epo_get_schedule(s.handle, 1)
    assert (ph[0], sw[0], st[0]) == (3, 2, 5)
    assert s.info().kernels_per_step == 4


def test_device_rule_equals_oracle_rule_on_a_real_sequence(ring8):
    sc, maps = ring8
    _, th0, _, _, _ = run_schedule(sc, maps, 40, sched_eps1=0.0, sched_w1=1000)
    eps1 = float(np.median(th0))  # crossed back and forth along this trajectory
    cfg = dict(sched_eps1=eps1, sched_w1=3, sched_eps2=0.5 * eps1, sched_w2=3)
    s, th, phases, th_o, frozen = run_schedule(sc, maps, 60, **cfg)
    assert np.allclose(th, th_o, rtol=1e-9, atol=1e-9)
    assert phases == oracle.converge_run(th, cfg["sched_eps1"], cfg["sched_w1"], cfg["sched_eps2"], cfg["sched_w2"])
    assert frozen


def test_schedule_off_and_argument_checks(ring8):
    sc, maps = ring8
    s = gpu_scene(sc, maps)
    with pytest.raises(epo.EpoError):
        B.epo_get_schedule(s.handle, 1)
    with pytest.raises(epo.EpoError):
        gpu_scene(sc, maps, schedule=1, sched_w1=0)
