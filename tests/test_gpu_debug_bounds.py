"""The debug build's gather bounds check (EPO_DEBUG_BOUNDS), the library's stand-in for a memory
sanitizer: every gather cell (x0, y0) must lie in [0, W - 2] x [0, H - 2]; a cell outside is
recorded, its fetch skipped, and the call returns EPO_ERR_INTERNAL naming the first offender,
with the poses left as they were.

Two variant builds run in child processes (the binding loads the build EPO_LIBRARY names):
  * the check as shipped: on valid inputs it never fires, and loss and gradient equal the
    release build's;
  * the check narrowed by 16 columns (EPO_DEBUG_BOUNDS_MARGIN=16), so that the report path runs
    on valid inputs: the last 16 cell columns count as outside, although every access stays
    inside the map (the check skips the fetch either way).
"""
import json
import os
import re
import subprocess
import sys

import numpy as np
import pytest

import synth
from tests.helpers import gpu_scene, grad_rel_err, oracle_maps_f32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA GPU required", allow_module_level=True)

import paper_2607_00579_gb300 as epo  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MARGIN = 16  # columns the narrowed check excludes at the right edge of every map

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import synth
import paper_2607_00579_gb300 as epo
from tests.helpers import gpu_scene, oracle_maps_f32
sc = synth.make_scene(synth.RING8_128x96)
s = gpu_scene(sc, oracle_maps_f32(sc))
s.set_poses(sc.T_init)
out = {}
for call in ("loss_and_grad", "again", "step"):
    try:
        if call == "step":
            s.step(1)
            out[call] = {"status": 0}
        else:
            loss, grad = s.loss_and_grad()
            out[call] = {"status": 0, "loss": float(loss[0]), "grad": grad.tolist()}
    except epo.EpoError as e:
        out[call] = {"status": e.status, "msg": str(e)}
out["poses_unchanged"] = bool(np.array_equal(s.get_poses(), np.asarray(sc.T_init).reshape(-1, 12)))
out["n_pairs"] = int(sc.n_pairs)
out["W"] = int(sc.W[0])
print(json.dumps(out))
"""


@pytest.fixture(scope="module")
def debug_builds(tmp_path_factory):
    d = tmp_path_factory.mktemp("epo_debug")
    libs = {}
    procs = []
    for name, defines in (("check", ["EPO_DEBUG_BOUNDS"]),
                          ("narrowed", ["EPO_DEBUG_BOUNDS", f"EPO_DEBUG_BOUNDS_MARGIN={MARGIN}"])):
        out = str(d / name / "libepo.so")
        os.makedirs(os.path.dirname(out), exist_ok=True)
        args = [sys.executable, "-m", "paper_2607_00579_gb300.build", "--out", out]
        for x in defines:
            args += ["--define", x]
        procs.append((name, out, subprocess.Popen(args, cwd=ROOT, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for name, out, p in procs:
        log, _ = p.communicate()
        assert p.returncode == 0, log.decode(errors="replace")[-2000:]
        libs[name] = out
    return libs


def run_child(lib):
    env = dict(os.environ, EPO_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_check_is_silent_on_valid_inputs_and_changes_nothing(debug_builds):
    out = run_child(debug_builds["check"])
    assert out["loss_and_grad"]["status"] == 0 and out["step"]["status"] == 0
    sc = synth.make_scene(synth.RING8_128x96)
    ref = gpu_scene(sc, oracle_maps_f32(sc))
    ref.set_poses(sc.T_init)
    loss, grad = ref.loss_and_grad()
    assert out["loss_and_grad"]["loss"] == pytest.approx(loss[0], rel=1e-12)
    assert grad_rel_err(np.array(out["loss_and_grad"]["grad"]), grad) < 1e-10


def test_narrowed_check_reports_internal_error_and_refuses_the_update(debug_builds):
    out = run_child(debug_builds["narrowed"])
    for call in ("loss_and_grad", "again", "step"):
        assert out[call]["status"] == epo._binding.EPO_ERR_INTERNAL, out[call]
    msg = out["loss_and_grad"]["msg"]
    m = re.search(r"gather cell outside its map \(pair (-?\d+), cell (-?\d+), (-?\d+)\)", msg)
    assert m, msg
    pair, x0, y0 = (int(g) for g in m.groups())
    # the first offender is a cell of the columns the narrowed check excludes
    assert out["W"] - 2 - MARGIN < x0 <= out["W"] - 2 and y0 >= 0
    assert 0 <= pair < out["n_pairs"]
    assert out["poses_unchanged"]
