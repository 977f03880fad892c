"""ctypes binding of libepo.so: the C ABI under the same names, argument marshalling only.

Every computation happens in the library's CUDA kernels; this module converts numpy
arrays / torch tensors to pointers and status codes to exceptions.  If the library is
missing or cannot be loaded the import of the functions raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libepo.so")

EPO_OK = 0
EPO_ERR_INVALID_ARG = 1
EPO_ERR_CUDA = 2
EPO_ERR_OOM = 3
EPO_ERR_NUMERIC = 4
EPO_ERR_TIMEOUT = 5
EPO_ERR_INTERNAL = 6
EPO_ERR_TOO_LARGE = 7
STATUS_NAMES = {0: "EPO_OK", 1: "EPO_ERR_INVALID_ARG", 2: "EPO_ERR_CUDA", 3: "EPO_ERR_OOM",
                4: "EPO_ERR_NUMERIC", 5: "EPO_ERR_TIMEOUT", 6: "EPO_ERR_INTERNAL",
                7: "EPO_ERR_TOO_LARGE"}
EPO_NOALLOC_MAX_VIEWS = 1024
EPO_NOALLOC_MAX_PAIRS = 4096

EPO_F32, EPO_F16, EPO_BF16 = 0, 1, 2
EPO_NORM_VALID, EPO_NORM_ALL = 0, 1
EPO_GATHER_AUTO, EPO_GATHER_LDG, EPO_GATHER_TEX, EPO_GATHER_MIX = 0, 1, 2, 3

# Every symbol declared in include/epo.h (checked by the test-suite).
EXPORTED = [
    "epo_default_options", "epo_abi_version", "epo_create_scene", "epo_create_batch",
    "epo_destroy_scene", "epo_last_error", "epo_scene_info_get", "epo_set_poses", "epo_get_poses",
    "epo_set_poses_dev", "epo_get_poses_dev", "epo_get_state", "epo_set_state", "epo_loss_and_grad",
    "epo_loss_and_grad_dev", "epo_pair_stats", "epo_forward_dev", "epo_backward_dev", "epo_step",
    "epo_step_async", "epo_step_plain", "epo_check", "epo_set_pair_subset", "epo_autotune",
    "epo_distance_field", "epo_round_bf16", "epo_last_loss", "epo_kernel_time", "epo_fixup_stats", "epo_stage_times",
    "epo_loss_and_grad_noalloc", "epo_gather_probe", "epo_set_refinement", "epo_refine_loss_and_grad",
    "epo_get_pair_active", "epo_get_schedule", "epo_build_viewgraph", "epo_get_refinement",
    "epo_set_pose_mlp", "epo_get_pose_mlp", "epo_get_pose_mlp_moments", "epo_step_host",
    "epo_set_wait_limit",
]


class EpoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class epo_view_desc(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int32), ("H", ctypes.c_int32), ("fx", ctypes.c_double),
                ("fy", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("records", ctypes.c_void_p), ("n_records", ctypes.c_int64), ("map", ctypes.c_void_p)]


class epo_scene_desc(ctypes.Structure):
    _fields_ = [("n_views", ctypes.c_int32), ("views", ctypes.POINTER(epo_view_desc)),
                ("n_pairs", ctypes.c_int32), ("pairs", ctypes.c_void_p), ("fixed", ctypes.c_void_p),
                ("record_dtype", ctypes.c_int32), ("map_dtype", ctypes.c_int32),
                ("pointers_on_device", ctypes.c_int32)]


class epo_options(ctypes.Structure):
    _fields_ = [("huber_delta", ctypes.c_double), ("lambda0", ctypes.c_double),
                ("lambda1", ctypes.c_double), ("lambda_steps", ctypes.c_int32),
                ("eps_z", ctypes.c_double), ("norm_mode", ctypes.c_int32),
                ("lr_rot", ctypes.c_double), ("lr_trans", ctypes.c_double),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("adam_eps", ctypes.c_double),
                ("autotune", ctypes.c_int32), ("gather", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("records_per_thread", ctypes.c_int32),
                ("grid_blocks", ctypes.c_int32), ("timing", ctypes.c_int32), ("tail_pairs", ctypes.c_int32),
                ("refine", ctypes.c_int32), ("pair_budget", ctypes.c_int32),
                ("subsample_seed", ctypes.c_uint64), ("sched_eps1", ctypes.c_double),
                ("sched_eps2", ctypes.c_double), ("schedule", ctypes.c_int32), ("sched_w1", ctypes.c_int32),
                ("sched_w2", ctypes.c_int32), ("lr_focal", ctypes.c_double), ("lr_depth", ctypes.c_double),
                ("pose_param", ctypes.c_int32), ("mlp_lr", ctypes.c_double), ("mlp_warmup", ctypes.c_int32),
                ("mlp_steps", ctypes.c_int32), ("mlp_wd", ctypes.c_double), ("mlp_wd_delta", ctypes.c_double),
                ("mlp_eps", ctypes.c_double)]


class epo_scene_info(ctypes.Structure):
    _fields_ = [("n_scenes", ctypes.c_int32), ("n_views", ctypes.c_int32), ("n_pairs", ctypes.c_int32),
                ("n_records", ctypes.c_int64), ("n_dropped", ctypes.c_int64),
                ("evals_per_step", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("record_bytes", ctypes.c_int64), ("map_bytes", ctypes.c_int64),
                ("n_tiles", ctypes.c_int32), ("gather", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("records_per_thread", ctypes.c_int32),
                ("grid_blocks", ctypes.c_int32), ("kernels_per_step", ctypes.c_int32),
                ("tail_pairs", ctypes.c_int32)]


class epo_noalloc_problem(ctypes.Structure):
    _fields_ = [("n_views", ctypes.c_int32), ("n_pairs", ctypes.c_int32), ("records", ctypes.c_void_p),
                ("rec_off", ctypes.c_void_p), ("max_records_per_view", ctypes.c_int64),
                ("maps", ctypes.c_void_p), ("map_off", ctypes.c_void_p), ("W", ctypes.c_void_p),
                ("H", ctypes.c_void_p), ("K", ctypes.c_void_p), ("pairs", ctypes.c_void_p),
                ("T", ctypes.c_void_p), ("lam", ctypes.c_double), ("huber_delta", ctypes.c_double),
                ("eps_z", ctypes.c_double), ("norm_mode", ctypes.c_int32)]


_lib = None


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libepo.so (building it with nvcc first if it is missing or stale), or the build
    that the environment variable EPO_LIBRARY names (a variant built by build.py --out)."""
    global _lib
    if _lib is not None:
        return _lib
    path = os.environ.get("EPO_LIBRARY") or LIB_PATH
    if build_if_missing and path == LIB_PATH:
        from . import build as _b
        _b.build()
    if not os.path.exists(path):
        raise ImportError(f"libepo.so not built at {path}")
    lib = ctypes.CDLL(path)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    S = ctypes.c_void_p  # epo_scene_t
    sig = {
        "epo_default_options": (None, [ctypes.POINTER(epo_options)]),
        "epo_abi_version": (I32, []),
        "epo_create_scene": (I32, [ctypes.POINTER(epo_scene_desc), ctypes.POINTER(epo_options), P,
                                   ctypes.POINTER(S)]),
        "epo_create_batch": (I32, [I32, ctypes.POINTER(epo_scene_desc), ctypes.POINTER(epo_options), P,
                                   ctypes.POINTER(S)]),
        "epo_destroy_scene": (None, [S]),
        "epo_last_error": (ctypes.c_char_p, [S]),
        "epo_scene_info_get": (I32, [S, ctypes.POINTER(epo_scene_info)]),
        "epo_set_poses": (I32, [S, P]),
        "epo_get_poses": (I32, [S, P]),
        "epo_set_poses_dev": (I32, [S, P]),
        "epo_get_poses_dev": (I32, [S, P]),
        "epo_get_state": (I32, [S, P, P, P]),
        "epo_set_state": (I32, [S, I64, P, P]),
        "epo_loss_and_grad": (I32, [S, P, P]),
        "epo_loss_and_grad_dev": (I32, [S, P, P]),
        "epo_pair_stats": (I32, [S, P]),
        "epo_forward_dev": (I32, [S, P, P]),
        "epo_backward_dev": (I32, [S, P, P, P]),
        "epo_step": (I32, [S, I32]),
        "epo_step_async": (I32, [S, I32]),
        "epo_step_plain": (I32, [S, I32]),
        "epo_check": (I32, [S]),
        "epo_set_wait_limit": (I32, [S, D]),
        "epo_set_pair_subset": (I32, [S, I32, P]),
        "epo_autotune": (I32, [S]),
        "epo_distance_field": (I32, [P, I32, I32, P, P]),
        "epo_round_bf16": (I32, [P, P, I64, P]),
        "epo_last_loss": (I32, [S, P]),
        "epo_kernel_time": (I32, [S, ctypes.POINTER(ctypes.c_float)]),
        "epo_fixup_stats": (I32, [S, P, P]),
        "epo_stage_times": (I32, [S, P]),
        "epo_loss_and_grad_noalloc": (I32, [ctypes.POINTER(epo_noalloc_problem), P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def check(status: int, scene=None) -> None:
    if status != EPO_OK:
        msg = load().epo_last_error(scene)
        raise EpoError(status, msg.decode() if msg else "")


def default_options(**overrides) -> epo_options:
    o = epo_options()
    load().epo_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


# ---- the C names, marshalled ----
def _ptr(x):
    """Pointer of a numpy array, a torch tensor or an int/None."""
    if x is None:
        return None
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    if hasattr(x, "ctypes"):
        return ctypes.c_void_p(x.ctypes.data)
    raise TypeError(type(x))


def epo_abi_version() -> int:
    return load().epo_abi_version()


def epo_create_batch(descs, opts, stream: int = 0) -> ctypes.c_void_p:
    arr = (epo_scene_desc * len(descs))(*descs)
    out = ctypes.c_void_p()
    st = load().epo_create_batch(len(descs), arr, ctypes.byref(opts), ctypes.c_void_p(stream),
                                 ctypes.byref(out))
    check(st, None)
    return out


def epo_create_scene(desc, opts, stream: int = 0) -> ctypes.c_void_p:
    out = ctypes.c_void_p()
    st = load().epo_create_scene(ctypes.byref(desc), ctypes.byref(opts), ctypes.c_void_p(stream),
                                 ctypes.byref(out))
    check(st, None)
    return out


def epo_destroy_scene(scene) -> None:
    load().epo_destroy_scene(scene)


def epo_scene_info_get(scene) -> epo_scene_info:
    info = epo_scene_info()
    check(load().epo_scene_info_get(scene, ctypes.byref(info)), scene)
    return info


def _call(name, scene, *args):
    check(getattr(load(), name)(scene, *args), scene)


def epo_set_poses(scene, T): _call("epo_set_poses", scene, _ptr(T))
def epo_get_poses(scene, T): _call("epo_get_poses", scene, _ptr(T))
def epo_set_poses_dev(scene, T): _call("epo_set_poses_dev", scene, _ptr(T))
def epo_get_poses_dev(scene, T): _call("epo_get_poses_dev", scene, _ptr(T))
def epo_get_state(scene, step_arr, m, v): _call("epo_get_state", scene, _ptr(step_arr), _ptr(m), _ptr(v))
def epo_set_state(scene, step, m, v): _call("epo_set_state", scene, ctypes.c_int64(step), _ptr(m), _ptr(v))
def epo_loss_and_grad(scene, loss, grad): _call("epo_loss_and_grad", scene, _ptr(loss), _ptr(grad))
def epo_loss_and_grad_dev(scene, loss, grad): _call("epo_loss_and_grad_dev", scene, _ptr(loss), _ptr(grad))
def epo_pair_stats(scene, stats): _call("epo_pair_stats", scene, _ptr(stats))
def epo_forward_dev(scene, xi, loss): _call("epo_forward_dev", scene, _ptr(xi), _ptr(loss))
def epo_backward_dev(scene, xi, dloss, grad): _call("epo_backward_dev", scene, _ptr(xi), _ptr(dloss), _ptr(grad))
def epo_step(scene, n): _call("epo_step", scene, ctypes.c_int32(n))
def epo_step_async(scene, n): _call("epo_step_async", scene, ctypes.c_int32(n))
def epo_step_plain(scene, n): _call("epo_step_plain", scene, ctypes.c_int32(n))
def epo_check(scene): _call("epo_check", scene)
def epo_set_wait_limit(scene, seconds: float): _call("epo_set_wait_limit", scene, float(seconds))
def epo_autotune(scene): _call("epo_autotune", scene)
def epo_last_loss(scene, loss): _call("epo_last_loss", scene, _ptr(loss))


def epo_fixup_stats(scene):
    q = ctypes.c_int64(0)
    o = ctypes.c_int64(0)
    _call("epo_fixup_stats", scene, ctypes.byref(q), ctypes.byref(o))
    return int(q.value), int(o.value)


def epo_stage_times(scene):
    ms = (ctypes.c_float * 3)()
    _call("epo_stage_times", scene, ms)
    return [float(x) for x in ms]


def epo_kernel_time(scene) -> float:
    ms = ctypes.c_float(0.0)
    _call("epo_kernel_time", scene, ctypes.byref(ms))
    return float(ms.value)


def epo_set_pair_subset(scene, ids):
    import numpy as np
    a = np.ascontiguousarray(ids, dtype=np.int32) if ids is not None and len(ids) else None
    _call("epo_set_pair_subset", scene, ctypes.c_int32(0 if a is None else len(a)), _ptr(a))


def epo_loss_and_grad_noalloc(problem, loss_dev, grad_dev, stream: int = 0) -> int:
    """Returns the status code (the caller decides how to report it)."""
    return load().epo_loss_and_grad_noalloc(ctypes.byref(problem), _ptr(loss_dev), _ptr(grad_dev),
                                            ctypes.c_void_p(stream))


def epo_distance_field(edges_dev, W: int, H: int, map_dev, stream: int = 0):
    check(load().epo_distance_field(_ptr(edges_dev), W, H, _ptr(map_dev), ctypes.c_void_p(stream)))


def epo_round_bf16(src_dev, dst_dev, n: int, stream: int = 0):
    check(load().epo_round_bf16(_ptr(src_dev), _ptr(dst_dev), ctypes.c_int64(n), ctypes.c_void_p(stream)))


def epo_get_schedule(scene, n_scenes: int):
    """Returns (theta95, phase, switch_step, stop_step), one entry per scene."""
    import numpy as np
    th = np.zeros(n_scenes)
    ph = np.zeros(n_scenes, dtype=np.int32)
    sw = np.zeros(n_scenes, dtype=np.int64)
    st = np.zeros(n_scenes, dtype=np.int64)
    _call("epo_get_schedule", scene, _ptr(th), _ptr(ph), _ptr(sw), _ptr(st))
    return th, ph, sw, st


def epo_get_pair_active(scene, n_pairs: int):
    import numpy as np
    out = np.zeros(max(n_pairs, 1), dtype=np.uint8)
    _call("epo_get_pair_active", scene, _ptr(out))
    return out[:n_pairs].astype(bool)


def epo_set_refinement(scene, gamma=None, alpha=None, beta=None):
    import numpy as np
    g = None if gamma is None else np.ascontiguousarray(gamma, dtype=np.float64)
    a = None if alpha is None else np.ascontiguousarray(alpha, dtype=np.float32)
    b = None if beta is None else np.ascontiguousarray(beta, dtype=np.float32)
    _call("epo_set_refinement", scene, _ptr(g), _ptr(a), _ptr(b))


EPO_POSE_SE3, EPO_POSE_MLP = 0, 1
EPO_POSE_MLP_PARAMS = 69260


def epo_set_pose_mlp(scene, params):
    import numpy as np
    p = np.ascontiguousarray(params, dtype=np.float32)
    _call("epo_set_pose_mlp", scene, _ptr(p))


def epo_get_pose_mlp(scene, n_scenes: int, n_views: int):
    """Returns (params (n_scenes, EPO_POSE_MLP_PARAMS) float32, delta (n_views, 3) float32)."""
    import numpy as np
    p = np.zeros((n_scenes, EPO_POSE_MLP_PARAMS), np.float32)
    d = np.zeros((n_views, 3), np.float32)
    _call("epo_get_pose_mlp", scene, _ptr(p), _ptr(d))
    return p, d


def epo_step_host(scene, T_in=None, T_out=None, loss=None):
    """One host-driven step (arrays: contiguous float64, pinned for asynchronous copies)."""
    _call("epo_step_host", scene, _ptr(T_in), _ptr(T_out), _ptr(loss))


def epo_get_pose_mlp_moments(scene, n_scenes: int, n_views: int):
    """Returns (m, v (n_scenes, EPO_POSE_MLP_PARAMS), dm, dv (n_views, 3)), float32."""
    import numpy as np
    m = np.zeros((n_scenes, EPO_POSE_MLP_PARAMS), np.float32)
    v = np.zeros_like(m)
    dm = np.zeros((n_views, 3), np.float32)
    dv = np.zeros_like(dm)
    _call("epo_get_pose_mlp_moments", scene, _ptr(m), _ptr(v), _ptr(dm), _ptr(dv))
    return m, v, dm, dv


def epo_get_refinement(scene, n_views: int, n_records: int):
    """Returns (gamma (n_views,) float64, alpha, beta (n_records,) float32)."""
    import numpy as np
    g = np.zeros(n_views)
    a = np.zeros(max(n_records, 1), np.float32)
    b = np.zeros(max(n_records, 1), np.float32)
    _call("epo_get_refinement", scene, _ptr(g), _ptr(a), _ptr(b))
    return g, a[:n_records], b[:n_records]


def epo_refine_loss_and_grad(scene, n_scenes: int, n_views: int, n_records: int):
    """Returns (loss (n_scenes,), grad (n_views, 6), grad_gamma (n_views,), grad_alpha, grad_beta
    (n_records,) float32)."""
    import numpy as np
    loss = np.zeros(n_scenes)
    grad = np.zeros((n_views, 6))
    gg = np.zeros(n_views)
    ga = np.zeros(max(n_records, 1), dtype=np.float32)
    gb = np.zeros(max(n_records, 1), dtype=np.float32)
    _call("epo_refine_loss_and_grad", scene, _ptr(loss), _ptr(grad), _ptr(gg), _ptr(ga), _ptr(gb))
    return loss, grad, gg, ga[:n_records], gb[:n_records]


def epo_build_viewgraph(W, H, K, T, depth_dev, stride: int, tau: float, min_frac: float, stream: int = 0):
    """Returns (frac (n, n), pairs (m, 2) int32)."""
    import numpy as np
    n = len(W)
    Wa = np.ascontiguousarray(W, dtype=np.int32)
    Ha = np.ascontiguousarray(H, dtype=np.int32)
    Ka = np.ascontiguousarray(K, dtype=np.float64).reshape(n, 4)
    Ta = np.ascontiguousarray(T, dtype=np.float64).reshape(n, 12)
    frac = np.zeros((n, n))
    pairs = np.zeros((max(n * (n - 1), 1), 2), dtype=np.int32)
    m = ctypes.c_int32(0)
    check(load().epo_build_viewgraph(ctypes.c_int32(n), _ptr(Wa), _ptr(Ha), _ptr(Ka), _ptr(Ta), _ptr(depth_dev),
                                     ctypes.c_int32(stride), ctypes.c_double(tau), ctypes.c_double(min_frac),
                                     _ptr(frac), _ptr(pairs), ctypes.byref(m), ctypes.c_void_p(stream)))
    return frac, pairs[:m.value]


def epo_gather_probe(n_maps: int, W: int, H: int, map_dtype: int, gather: int, pattern: int, samples: int,
                     repeats: int = 5, stream: int = 0) -> float:
    out = ctypes.c_double(0.0)
    check(load().epo_gather_probe(ctypes.c_int32(n_maps), ctypes.c_int32(W), ctypes.c_int32(H),
                                  ctypes.c_int32(map_dtype), ctypes.c_int32(gather), ctypes.c_int32(pattern),
                                  ctypes.c_int64(samples), ctypes.c_int32(repeats), ctypes.byref(out),
                                  ctypes.c_void_p(stream)))
    return out.value
