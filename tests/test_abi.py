"""The C-ABI library builds for sm_103a, loads, and exports every symbol its header declares.
Argument validation that returns before any CUDA call is checked here too (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_2607_00579_gb300 as epo
from paper_2607_00579_gb300 import _binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    src = open(os.path.join(ROOT, "include", "epo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(epo_[a-z0-9_]+)\s*\(", src)))


def test_library_loads_and_exports_every_declared_symbol():
    lib = B.load()
    names = header_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(B.EXPORTED) == names


def test_abi_version_and_defaults():
    assert epo._binding.epo_abi_version() == 4
    o = epo.default_options()
    assert o.huber_delta == 1.0 and o.lambda0 == 10.0 and o.lambda1 == 6.0 and o.lambda_steps == 1000
    assert o.beta1 == 0.9 and o.beta2 == 0.999 and o.norm_mode == epo.EPO_NORM_VALID


def test_invalid_arguments_return_status_without_a_gpu():
    lib = B.load()
    out = ctypes.c_void_p()
    o = epo.default_options()
    assert lib.epo_create_batch(0, None, ctypes.byref(o), None, ctypes.byref(out)) == B.EPO_ERR_INVALID_ARG
    assert lib.epo_create_scene(None, ctypes.byref(o), None, ctypes.byref(out)) == B.EPO_ERR_INVALID_ARG
    assert b"null" in lib.epo_last_error(None)
    # a view below the 2x2 minimum, an out-of-range pair, unknown dtypes: rejected before CUDA
    views = (B.epo_view_desc * 2)()
    for v in views:
        v.W, v.H, v.fx, v.fy, v.cx, v.cy = 1, 5, 1.0, 1.0, 0.0, 0.0
        v.map = 1
    pairs = (ctypes.c_int32 * 2)(0, 1)
    d = B.epo_scene_desc(2, ctypes.cast(views, ctypes.POINTER(B.epo_view_desc)), 1,
                         ctypes.cast(pairs, ctypes.c_void_p), None, 0, 0, 0)
    assert lib.epo_create_scene(ctypes.byref(d), ctypes.byref(o), None, ctypes.byref(out)) == B.EPO_ERR_INVALID_ARG
    for v in views:
        v.W = 4
    pairs[1] = 7
    assert lib.epo_create_scene(ctypes.byref(d), ctypes.byref(o), None, ctypes.byref(out)) == B.EPO_ERR_INVALID_ARG
    assert b"range" in lib.epo_last_error(None)
    pairs[1] = 1
    d.map_dtype = 9
    assert lib.epo_create_scene(ctypes.byref(d), ctypes.byref(o), None, ctypes.byref(out)) == B.EPO_ERR_INVALID_ARG
    d.map_dtype = 0
    bad = epo.default_options(records_per_thread=3)
    assert lib.epo_create_scene(ctypes.byref(d), ctypes.byref(bad), None, ctypes.byref(out)) == B.EPO_ERR_INVALID_ARG
    assert out.value is None
    # calls on a null handle
    assert lib.epo_loss_and_grad(None, None, None) == B.EPO_ERR_INVALID_ARG
    assert lib.epo_step(None, 1) == B.EPO_ERR_INVALID_ARG
    assert lib.epo_distance_field(None, 4, 4, None, None) == B.EPO_ERR_INVALID_ARG
    assert lib.epo_round_bf16(None, None, 4, None) == B.EPO_ERR_INVALID_ARG


def test_binding_raises_on_error_status():
    with pytest.raises(B.EpoError) as e:
        B.check(B.EPO_ERR_INVALID_ARG, None)
    assert e.value.status == B.EPO_ERR_INVALID_ARG
