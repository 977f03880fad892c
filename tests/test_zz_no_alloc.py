"""The entry point that allocates nothing, against the FP64 oracle and the scene entry point.

epo_loss_and_grad_noalloc serves callers that cannot call cudaMalloc (a host that owns all
device memory, a fixed memory budget, a real-time loop): they pass their own device
buffers, and the library keeps its intermediate sums in one fixed-size device array.
Two calls in a row, at different poses and under both per-direction normalisers, must each
agree with the oracle and with epo_loss_and_grad on the same inputs within the tolerances
of the parity tests; the second call also shows that the shared array is cleared between
calls.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import gpu_scene, grad_rel_err, oracle_maps_f32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA GPU required", allow_module_level=True)

from paper_2607_00579_gb300 import _binding as B  # noqa: E402
from tests.test_gpu_parity import check_against_oracle  # noqa: E402

LOSS_RTOL = 1e-5
GRAD_RTOL = 1e-4


class Problem:
    """A scene held in caller-owned device buffers, described by an epo_noalloc_problem."""

    def __init__(self, sc, maps, rec=None):
        dev = torch.device("cuda")
        rec = sc.rec if rec is None else rec
        self.records = torch.from_numpy(np.ascontiguousarray(rec)).to(dev)
        self.rec_off = torch.from_numpy(sc.rec_off.astype(np.int64)).to(dev)
        self.flat = torch.from_numpy(np.concatenate([m.reshape(-1) for m in maps])).to(dev)
        moff = np.concatenate([[0], np.cumsum([m.size for m in maps])[:-1]]).astype(np.int64)
        self.map_off = torch.from_numpy(moff).to(dev)
        self.W = torch.from_numpy(np.asarray(sc.W, dtype=np.int32)).to(dev)
        self.H = torch.from_numpy(np.asarray(sc.H, dtype=np.int32)).to(dev)
        self.K = torch.from_numpy(np.ascontiguousarray(sc.K, dtype=np.float64)).to(dev)
        self.pairs = torch.from_numpy(np.ascontiguousarray(np.asarray(sc.pairs).reshape(-1).astype(np.int32))).to(dev)
        self.T = torch.zeros((sc.n_views, 12), dtype=torch.float64, device=dev)
        self.loss = torch.zeros(1, dtype=torch.float64, device=dev)
        self.grad = torch.zeros((sc.n_views, 6), dtype=torch.float64, device=dev)
        p = B.epo_noalloc_problem()
        p.n_views, p.n_pairs = sc.n_views, len(sc.pairs)
        p.records, p.rec_off = self.records.data_ptr(), self.rec_off.data_ptr()
        p.max_records_per_view = int(np.diff(sc.rec_off).max())
        p.maps, p.map_off = self.flat.data_ptr(), self.map_off.data_ptr()
        p.W, p.H, p.K = self.W.data_ptr(), self.H.data_ptr(), self.K.data_ptr()
        p.pairs, p.T = self.pairs.data_ptr(), self.T.data_ptr()
        p.lam, p.huber_delta, p.eps_z = 10.0, 1.0, 1e-6
        p.norm_mode = B.EPO_NORM_VALID
        self.prob = p

    def __call__(self, poses, norm_mode):
        self.T.copy_(torch.from_numpy(np.ascontiguousarray(poses, dtype=np.float64)))
        self.prob.norm_mode = norm_mode
        st = B.epo_loss_and_grad_noalloc(self.prob, self.loss, self.grad, torch.cuda.current_stream().cuda_stream)
        assert st == B.EPO_OK, B.STATUS_NAMES.get(st, st)
        torch.cuda.synchronize()
        return float(self.loss.item()), self.grad.cpu().numpy()


@pytest.fixture(scope="module")
def ring8():
    sc = synth.make_scene(synth.RING8_128x96)
    return sc, oracle_maps_f32(sc)


@pytest.mark.parametrize("norm_mode", [B.EPO_NORM_VALID, B.EPO_NORM_ALL], ids=["norm-valid", "norm-all"])
def test_noalloc_matches_oracle_and_scene_entry_point_on_two_calls(ring8, norm_mode):
    sc, maps = ring8
    ref = gpu_scene(sc, maps, norm_mode=norm_mode)
    osc = oracle.scene_from_synth(sc, [m.astype(np.float64) for m in maps])
    onorm = oracle.NORM_ALL if norm_mode == B.EPO_NORM_ALL else oracle.NORM_VALID
    run = Problem(sc, maps)
    for poses in (sc.T_init, sc.T_gt):
        got_loss, got_grad = run(poses, norm_mode)
        # against the FP64 oracle, with the parity tests' tolerances and allowances
        o = osc.loss_grad(poses, lam=10.0, norm_mode=onorm)
        check_against_oracle(got_loss, got_grad, o, sc.pairs, poses)
        # against the scene entry point on the same inputs
        ref.set_poses(poses)
        want_loss, want_grad = ref.loss_and_grad()
        assert abs(got_loss - want_loss[0]) <= LOSS_RTOL * abs(want_loss[0]), (got_loss, want_loss[0])
        assert grad_rel_err(got_grad, want_grad) <= GRAD_RTOL


def test_noalloc_ignores_records_without_usable_depth(ring8):
    """Records whose depth is not positive are not part of the problem, as at scene creation:
    under Eq. 7's normaliser |E_i| counts only the usable records of view i."""
    sc, maps = ring8
    rec = sc.rec.copy()
    rng = np.random.default_rng(12)
    bad = rng.choice(len(rec), 40, replace=False)
    rec[bad, 2] = -1.0
    keep = np.ones(len(rec), bool)
    keep[bad] = False
    cnt = [int(keep[sc.rec_off[v]:sc.rec_off[v + 1]].sum()) for v in range(sc.n_views)]
    off = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
    osc = oracle.OracleScene(sc.W, sc.H, sc.K, off, sc.rec[keep], [m.astype(np.float64) for m in maps], sc.pairs)
    run = Problem(sc, maps, rec=rec)
    for norm_mode, onorm in ((B.EPO_NORM_VALID, oracle.NORM_VALID), (B.EPO_NORM_ALL, oracle.NORM_ALL)):
        got_loss, got_grad = run(sc.T_init, norm_mode)
        check_against_oracle(got_loss, got_grad, osc.loss_grad(sc.T_init, lam=10.0, norm_mode=onorm),
                             sc.pairs, sc.T_init)


def test_noalloc_rejects_problems_beyond_its_capacity_and_misaligned_buffers(ring8):
    sc, maps = ring8
    prob = B.epo_noalloc_problem()
    prob.n_views, prob.n_pairs = 8, B.EPO_NOALLOC_MAX_PAIRS + 1
    for name in ("records", "rec_off", "maps", "map_off", "W", "H", "K", "pairs", "T"):
        setattr(prob, name, 16)  # never dereferenced: the size checks come first
    prob.lam, prob.huber_delta, prob.eps_z = 10.0, 1.0, 1e-6
    out = torch.zeros(64, dtype=torch.float64, device="cuda")
    assert B.epo_loss_and_grad_noalloc(prob, out, out, 0) == B.EPO_ERR_TOO_LARGE
    prob.n_pairs, prob.n_views = 8, B.EPO_NOALLOC_MAX_VIEWS + 1
    assert B.epo_loss_and_grad_noalloc(prob, out, out, 0) == B.EPO_ERR_TOO_LARGE
    # more tiles of 256 records in one view than a grid dimension holds
    prob.n_views = 8
    prob.max_records_per_view = 256 * (2 ** 31)
    assert B.epo_loss_and_grad_noalloc(prob, out, out, 0) == B.EPO_ERR_TOO_LARGE
    # records read as 16-byte vectors: a pointer off that boundary is refused before any launch
    run = Problem(sc, maps)
    good = run.prob.records
    run.prob.records = good + 4
    assert B.epo_loss_and_grad_noalloc(run.prob, run.loss, run.grad, 0) == B.EPO_ERR_INVALID_ARG
    run.prob.records = good
    run.prob.T = run.T.data_ptr() + 4
    assert B.epo_loss_and_grad_noalloc(run.prob, run.loss, run.grad, 0) == B.EPO_ERR_INVALID_ARG
    run.prob.T = run.T.data_ptr()
    # and the problem still runs afterwards
    got_loss, _ = run(sc.T_init, B.EPO_NORM_VALID)
    assert np.isfinite(got_loss) and got_loss > 0
