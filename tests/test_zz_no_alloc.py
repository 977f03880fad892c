"""The entry point that allocates nothing, against the scene-based entry point.

epo_loss_and_grad_noalloc serves callers that cannot call cudaMalloc (a host that owns all
device memory, a fixed memory budget, a real-time loop): they pass their own device
buffers, and the library keeps its intermediate sums in one fixed-size device array.
Two calls in a row, at different poses, must each agree with epo_loss_and_grad on the
same inputs within the tolerances of the parity tests; the second call also shows that
the shared array is cleared between calls.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import synth
from tests.helpers import gpu_scene, grad_rel_err, oracle_maps_f32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA GPU required", allow_module_level=True)

from paper_2607_00579_gb300 import _binding as B  # noqa: E402

LOSS_RTOL = 1e-5
GRAD_RTOL = 1e-4


def test_noalloc_matches_scene_entry_point_on_two_calls():
    sc = synth.make_scene(synth.RING8_128x96)
    maps = oracle_maps_f32(sc)
    ref = gpu_scene(sc, maps)

    dev = torch.device("cuda")
    records = torch.from_numpy(np.ascontiguousarray(sc.rec)).to(dev)
    rec_off = torch.from_numpy(sc.rec_off.astype(np.int64)).to(dev)
    flat = torch.from_numpy(np.concatenate([m.reshape(-1) for m in maps])).to(dev)
    moff = np.concatenate([[0], np.cumsum([m.size for m in maps])[:-1]]).astype(np.int64)
    map_off = torch.from_numpy(moff).to(dev)
    W = torch.from_numpy(sc.W.astype(np.int32)).to(dev)
    H = torch.from_numpy(sc.H.astype(np.int32)).to(dev)
    K = torch.from_numpy(np.ascontiguousarray(sc.K)).to(dev)
    pairs = torch.from_numpy(np.ascontiguousarray(sc.pairs.reshape(-1).astype(np.int32))).to(dev)
    T = torch.zeros((sc.n_views, 12), dtype=torch.float64, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    grad = torch.zeros((sc.n_views, 6), dtype=torch.float64, device=dev)

    prob = B.epo_noalloc_problem()
    prob.n_views, prob.n_pairs = sc.n_views, sc.n_pairs
    prob.records, prob.rec_off = records.data_ptr(), rec_off.data_ptr()
    prob.max_records_per_view = int(np.diff(sc.rec_off).max())
    prob.maps, prob.map_off = flat.data_ptr(), map_off.data_ptr()
    prob.W, prob.H, prob.K = W.data_ptr(), H.data_ptr(), K.data_ptr()
    prob.pairs, prob.T = pairs.data_ptr(), T.data_ptr()
    prob.lam, prob.huber_delta, prob.eps_z = 10.0, 1.0, 1e-6
    prob.norm_mode = B.EPO_NORM_VALID
    stream = torch.cuda.current_stream().cuda_stream

    for poses in (sc.T_init, sc.T_gt):
        ref.set_poses(poses)
        want_loss, want_grad = ref.loss_and_grad()
        T.copy_(torch.from_numpy(np.ascontiguousarray(poses)))
        st = B.epo_loss_and_grad_noalloc(prob, loss, grad, stream)
        assert st == B.EPO_OK, B.STATUS_NAMES.get(st, st)
        torch.cuda.synchronize()
        got_loss = float(loss.item())
        assert abs(got_loss - want_loss[0]) <= LOSS_RTOL * abs(want_loss[0]), (got_loss, want_loss[0])
        assert grad_rel_err(grad.cpu().numpy(), want_grad) <= GRAD_RTOL


def test_noalloc_rejects_problems_beyond_its_capacity():
    prob = B.epo_noalloc_problem()
    prob.n_views, prob.n_pairs = 8, B.EPO_NOALLOC_MAX_PAIRS + 1
    for name in ("records", "rec_off", "maps", "map_off", "W", "H", "K", "pairs", "T"):
        setattr(prob, name, 16)  # never dereferenced: the size check comes first
    prob.lam, prob.huber_delta, prob.eps_z = 10.0, 1.0, 1e-6
    out = torch.zeros(64, dtype=torch.float64, device="cuda")
    assert B.epo_loss_and_grad_noalloc(prob, out, out, 0) == B.EPO_ERR_TOO_LARGE
    prob.n_pairs, prob.n_views = 8, B.EPO_NOALLOC_MAX_VIEWS + 1
    assert B.epo_loss_and_grad_noalloc(prob, out, out, 0) == B.EPO_ERR_TOO_LARGE
