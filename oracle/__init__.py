"""EPO FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Thin ctypes wrapper over ``epo_oracle.c`` (plain C, double precision, OpenMP over
pairs with a fixed-order final reduction).  Only ``tests/``, the smoke check and the
CPU-baseline leg of ``bench.py`` may import this package; the CUDA library and its
Python binding never do.

What it computes (Section 3 and the appendix algorithms):
  * ``edt`` / ``edt_brute``: the distance transform field DTF_i (Algorithm 1,
    ComputeDistanceFields), exact L2 (Felzenszwalb-Huttenlocher) and brute force;
  * ``loss_grad``: the edge reprojection loss (Eqs. 6-8) with per-pair statistics and
    the analytic left-perturbation pose gradient;
  * ``optimize``: the optimisation loop of Algorithm 2 restricted to poses (lambda
    anneal of Algorithm 3, tangent-space Adam, Exp retraction);
  * ``se3_exp`` / ``se3_log`` / ``se3_left_jacobian`` and ``robust``.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "epo_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_epo_oracle.so")
_lib = None

NORM_VALID = 0
NORM_ALL = 1


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Scene(ctypes.Structure):
    _fields_ = [("n_views", ctypes.c_int), ("W", ctypes.c_void_p), ("H", ctypes.c_void_p),
                ("K", ctypes.c_void_p), ("rec_off", ctypes.c_void_p), ("rec", ctypes.c_void_p),
                ("map_off", ctypes.c_void_p), ("map", ctypes.c_void_p), ("n_pairs", ctypes.c_int),
                ("pairs", ctypes.c_void_p)]


class _Params(ctypes.Structure):
    _fields_ = [("lam", ctypes.c_double), ("delta", ctypes.c_double), ("eps_z", ctypes.c_double),
                ("norm_mode", ctypes.c_int), ("near_margin", ctypes.c_double)]


class _Opt(ctypes.Structure):
    _fields_ = [("lambda0", ctypes.c_double), ("lambda1", ctypes.c_double),
                ("lambda_steps", ctypes.c_int), ("delta", ctypes.c_double),
                ("eps_z", ctypes.c_double), ("norm_mode", ctypes.c_int),
                ("lr_rot", ctypes.c_double), ("lr_trans", ctypes.c_double),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("eps", ctypes.c_double),
                ("pair_budget", ctypes.c_int), ("seed", ctypes.c_uint64)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        lib.oracle_edt.argtypes = [P, ctypes.c_int, ctypes.c_int, P]
        lib.oracle_edt_brute.argtypes = [P, ctypes.c_int, ctypes.c_int, P]
        lib.oracle_robust.argtypes = [ctypes.c_double] * 3 + [P, P]
        lib.oracle_robust.restype = None
        lib.oracle_loss_grad.argtypes = [P, P, P, P, P, P, P, P, P, P]
        lib.oracle_se3_exp.argtypes = [P, P]
        lib.oracle_se3_exp.restype = None
        lib.oracle_se3_log.argtypes = [P, P]
        lib.oracle_se3_log.restype = None
        lib.oracle_se3_left_jacobian.argtypes = [P, P]
        lib.oracle_se3_left_jacobian.restype = None
        lib.oracle_lambda.argtypes = [P, ctypes.c_int64]
        lib.oracle_lambda.restype = ctypes.c_double
        lib.oracle_optimize.argtypes = [P, P, P, P, ctypes.c_int64, ctypes.c_int, P, P, P]
        lib.oracle_loss_grad_full.argtypes = [P] * 11
        lib.oracle_splitmix64.argtypes = [ctypes.c_uint64]
        lib.oracle_splitmix64.restype = ctypes.c_uint64
        lib.oracle_pair_key.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32]
        lib.oracle_pair_key.restype = ctypes.c_uint64
        lib.oracle_subsample.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, P]
        lib.oracle_pose_change.argtypes = [P, P, ctypes.c_int, P, P]
        lib.oracle_pose_change.restype = None
        lib.oracle_percentile.argtypes = [P, ctypes.c_int, ctypes.c_double]
        lib.oracle_percentile.restype = ctypes.c_double
        lib.oracle_theta95.argtypes = [P, P, ctypes.c_int]
        lib.oracle_theta95.restype = ctypes.c_double
        lib.oracle_converge_update.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                               ctypes.c_int]
        lib.oracle_viewgraph.argtypes = [ctypes.c_int, P, P, P, P, P, ctypes.c_int, ctypes.c_double, P]
        lib.oracle_refine_step.argtypes = [P] * 7 + [ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                                     ctypes.c_double] + [P] * 9
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


# ----------------------------------------------------------------------------------------
def edt(edge: np.ndarray) -> np.ndarray:
    """Exact Euclidean distance (pixels) to the nearest nonzero pixel of ``edge`` (H, W)."""
    e = np.ascontiguousarray(edge, dtype=np.uint8)
    H, W = e.shape
    out = np.empty((H, W), dtype=np.float64)
    rc = _load().oracle_edt(_p(e), W, H, _p(out))
    if rc:
        raise RuntimeError(f"oracle_edt failed ({rc})")
    return out


def edt_brute(edge: np.ndarray) -> np.ndarray:
    e = np.ascontiguousarray(edge, dtype=np.uint8)
    H, W = e.shape
    out = np.empty((H, W), dtype=np.float64)
    _load().oracle_edt_brute(_p(e), W, H, _p(out))
    return out


def robust(d: float, lam: float, delta: float):
    """(rho, drho) = (H_delta(min(d, lambda)), gradient passed through the clamp)."""
    r = np.zeros(1)
    g = np.zeros(1)
    _load().oracle_robust(float(d), float(lam), float(delta), _p(r), _p(g))
    return float(r[0]), float(g[0])


def se3_exp(xi) -> np.ndarray:
    x = np.ascontiguousarray(xi, dtype=np.float64).reshape(6)
    T = np.zeros(12)
    _load().oracle_se3_exp(_p(x), _p(T))
    return T


def se3_log(T) -> np.ndarray:
    t = np.ascontiguousarray(T, dtype=np.float64).reshape(12)
    xi = np.zeros(6)
    _load().oracle_se3_log(_p(t), _p(xi))
    return xi


def se3_left_jacobian(xi) -> np.ndarray:
    x = np.ascontiguousarray(xi, dtype=np.float64).reshape(6)
    J = np.zeros(36)
    _load().oracle_se3_left_jacobian(_p(x), _p(J))
    return J.reshape(6, 6)


class OracleScene:
    """Scene in the oracle's flat FP64 layout.

    rec: (n_rec, >=3) (u, v, z) -- pass the values the GPU stores (already rounded).
    maps: list of (H, W) arrays -- pass the values the GPU stores (already rounded).
    """

    def __init__(self, W: Sequence[int], H: Sequence[int], K: np.ndarray, rec_off: np.ndarray,
                 rec: np.ndarray, maps: Sequence[np.ndarray], pairs: np.ndarray):
        self.W = np.ascontiguousarray(W, dtype=np.int32)
        self.H = np.ascontiguousarray(H, dtype=np.int32)
        self.K = np.ascontiguousarray(K, dtype=np.float64).reshape(-1, 4)
        self.rec_off = np.ascontiguousarray(rec_off, dtype=np.int64)
        self.rec = np.ascontiguousarray(np.asarray(rec, dtype=np.float64)[:, :3])
        self.map_off = np.zeros(len(maps), dtype=np.int64)
        off = 0
        for v, m in enumerate(maps):
            self.map_off[v] = off
            off += m.size
        self.map = np.ascontiguousarray(np.concatenate([np.asarray(m, np.float64).reshape(-1) for m in maps])
                                        if maps else np.zeros(1))
        self.pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        self.n_views = len(self.W)
        self.n_pairs = self.pairs.shape[0]
        self._s = _Scene(self.n_views, self.W.ctypes.data, self.H.ctypes.data, self.K.ctypes.data,
                         self.rec_off.ctypes.data, self.rec.ctypes.data, self.map_off.ctypes.data,
                         self.map.ctypes.data, self.n_pairs, self.pairs.ctypes.data)

    def loss_grad(self, T: np.ndarray, lam: float, delta: float = 1.0, eps_z: float = 1e-6,
                  norm_mode: int = NORM_VALID, near_margin: float = 1e-9):
        """Returns dict(loss, grad (n,6), pair_stats (P,8), pair_near (P,), pair_loss (P,),
        pair_abs (P,6), pair_maxterm (P,)).

        pair_near counts the samples whose position lies within near_margin pixels of the
        image border (or whose depth lies that close to eps_z): there the validity decision
        depends on the rounding of the arithmetic, not only on the mathematics."""
        T = np.ascontiguousarray(T, dtype=np.float64).reshape(self.n_views, 12)
        prm = _Params(lam, delta, eps_z, norm_mode, near_margin)
        loss = np.zeros(1)
        grad = np.zeros((self.n_views, 6))
        P = max(self.n_pairs, 1)
        st = np.zeros((P, 8))
        near = np.zeros(P, dtype=np.int64)
        pl = np.zeros(P)
        ab = np.zeros((P, 6))
        mt = np.zeros(P)
        rc = _load().oracle_loss_grad(ctypes.byref(self._s), _p(T), ctypes.byref(prm), _p(loss), _p(grad),
                                      _p(st), _p(near), _p(pl), _p(ab), _p(mt))
        if rc:
            raise ValueError(f"oracle_loss_grad failed ({rc})")
        return dict(loss=float(loss[0]), grad=grad, pair_stats=st[:self.n_pairs],
                    pair_near=near[:self.n_pairs], pair_loss=pl[:self.n_pairs], pair_abs=ab[:self.n_pairs],
                    pair_maxterm=mt[:self.n_pairs])

    def loss_grad_full(self, T: np.ndarray, gamma: np.ndarray, alpha: np.ndarray, beta: np.ndarray, lam: float,
                       delta: float = 1.0, eps_z: float = 1e-6, norm_mode: int = NORM_VALID):
        """Objective with focal scales gamma (per view, f = f0 (1 + gamma)) and per-record depth
        parameters (z = z0 alpha + beta).  Returns dict(loss, grad (n,6), grad_gamma (n,),
        grad_alpha (n_rec,), grad_beta (n_rec,))."""
        T = np.ascontiguousarray(T, dtype=np.float64).reshape(self.n_views, 12)
        g = np.ascontiguousarray(gamma, dtype=np.float64).reshape(self.n_views)
        n_rec = self.rec.shape[0]
        a = np.ascontiguousarray(alpha, dtype=np.float64).reshape(n_rec)
        b = np.ascontiguousarray(beta, dtype=np.float64).reshape(n_rec)
        prm = _Params(lam, delta, eps_z, norm_mode, 1e-9)
        loss = np.zeros(1)
        grad = np.zeros((self.n_views, 6))
        gg = np.zeros(self.n_views)
        ga = np.zeros(max(n_rec, 1))
        gb = np.zeros(max(n_rec, 1))
        rc = _load().oracle_loss_grad_full(ctypes.byref(self._s), _p(T), _p(g), _p(a), _p(b), ctypes.byref(prm),
                                           _p(loss), _p(grad), _p(gg), _p(ga), _p(gb))
        if rc:
            raise ValueError(f"oracle_loss_grad_full failed ({rc})")
        return dict(loss=float(loss[0]), grad=grad, grad_gamma=gg, grad_alpha=ga[:n_rec], grad_beta=gb[:n_rec])

    def refine_step(self, state: dict, fixed: np.ndarray, step: int, depth_t: int, lr_focal: float, lr_depth: float,
                    *, lambda0=10.0, lambda1=6.0, lambda_steps=1000, delta=1.0, eps_z=1e-6, norm_mode=NORM_VALID,
                    lr_rot=1e-3, lr_trans=1e-2, beta1=0.9, beta2=0.999, eps=1e-12) -> float:
        """One step of the full refinement on `state` (dict of T, gamma, alpha, beta and their Adam
        moments m, v, mg, vg, ma, va, mb, vb; created with refine_state), updated in place.
        Returns the loss before the step."""
        opt = _Opt(lambda0, lambda1, lambda_steps, delta, eps_z, norm_mode, lr_rot, lr_trans, beta1, beta2, eps, 0, 0)
        fx = np.ascontiguousarray(fixed, dtype=np.uint8)
        loss = np.zeros(1)
        st = state
        rc = _load().oracle_refine_step(ctypes.byref(self._s), _p(st["T"]), _p(st["gamma"]), _p(st["alpha"]),
                                        _p(st["beta"]), _p(fx), ctypes.byref(opt), int(step), int(depth_t),
                                        float(lr_focal), float(lr_depth), _p(st["m"]), _p(st["v"]), _p(st["mg"]),
                                        _p(st["vg"]), _p(st["ma"]), _p(st["va"]), _p(st["mb"]), _p(st["vb"]),
                                        _p(loss))
        if rc:
            raise ValueError(f"oracle_refine_step failed ({rc})")
        return float(loss[0])

    def refine_state(self, T, gamma, alpha, beta) -> dict:
        n, r = self.n_views, self.rec.shape[0]
        c = lambda x, k: np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(k), dtype=np.float64).copy()
        return dict(T=c(T, n * 12).reshape(n, 12), gamma=c(gamma, n), alpha=c(alpha, r), beta=c(beta, r),
                    m=np.zeros((n, 6)), v=np.zeros((n, 6)), mg=np.zeros(n), vg=np.zeros(n), ma=np.zeros(r),
                    va=np.zeros(r), mb=np.zeros(r), vb=np.zeros(r))

    def optimize(self, T: np.ndarray, fixed: np.ndarray, n_steps: int, *, lambda0=10.0, lambda1=6.0,
                 lambda_steps=1000, delta=1.0, eps_z=1e-6, norm_mode=NORM_VALID, lr_rot=1e-3,
                 lr_trans=1e-2, beta1=0.9, beta2=0.999, eps=1e-12, step0=0, m=None, v=None, pair_budget=0,
                 seed=0):
        """Run n_steps of Algorithm 2 (pose-only, tangent-space Adam).  Returns (T, m, v, losses)."""
        T = np.ascontiguousarray(T, dtype=np.float64).reshape(self.n_views, 12).copy()
        fx = np.ascontiguousarray(fixed, dtype=np.uint8)
        m = np.zeros((self.n_views, 6)) if m is None else np.ascontiguousarray(m, np.float64).copy()
        v = np.zeros((self.n_views, 6)) if v is None else np.ascontiguousarray(v, np.float64).copy()
        hist = np.zeros(max(n_steps, 1))
        opt = _Opt(lambda0, lambda1, lambda_steps, delta, eps_z, norm_mode, lr_rot, lr_trans, beta1,
                   beta2, eps, pair_budget, seed & (2**64 - 1))
        rc = _load().oracle_optimize(ctypes.byref(self._s), _p(T), _p(fx), ctypes.byref(opt), step0,
                                     n_steps, _p(m), _p(v), _p(hist))
        if rc:
            raise ValueError(f"oracle_optimize failed ({rc})")
        return T, m, v, hist[:n_steps]


def splitmix64(state: int) -> int:
    """SplitMix64's output for a state (the increment added first)."""
    return int(_load().oracle_splitmix64(ctypes.c_uint64(state & (2**64 - 1))))


def pair_key(seed: int, step: int, p: int) -> int:
    return int(_load().oracle_pair_key(ctypes.c_uint64(seed & (2**64 - 1)), step, p))


def subsample(seed: int, step: int, n_pairs: int, M: int) -> np.ndarray:
    """Pairs of one scene evaluated at a step (Algorithm 3's fresh uniform subset of
    min(|E|, M)): boolean mask over the scene's pairs."""
    out = np.zeros(max(n_pairs, 1), dtype=np.uint8)
    rc = _load().oracle_subsample(ctypes.c_uint64(seed & (2**64 - 1)), step, n_pairs, M, _p(out))
    if rc:
        raise ValueError(f"oracle_subsample failed ({rc})")
    return out[:n_pairs].astype(bool)


def pose_change(T_prev, T_new):
    """Per-view rotation and translation-direction change in degrees (Section 3)."""
    A = np.ascontiguousarray(T_prev, dtype=np.float64).reshape(-1, 12)
    Bn = np.ascontiguousarray(T_new, dtype=np.float64).reshape(-1, 12)
    n = A.shape[0]
    dR, dt = np.zeros(n), np.zeros(n)
    _load().oracle_pose_change(_p(A), _p(Bn), n, _p(dR), _p(dt))
    return dR, dt


def percentile(x, q: float) -> float:
    a = np.ascontiguousarray(x, dtype=np.float64)
    return float(_load().oracle_percentile(_p(a), a.size, q))


def theta95(T_prev, T_new) -> float:
    A = np.ascontiguousarray(T_prev, dtype=np.float64).reshape(-1, 12)
    Bn = np.ascontiguousarray(T_new, dtype=np.float64).reshape(-1, 12)
    return float(_load().oracle_theta95(_p(A), _p(Bn), A.shape[0]))


def converge_run(thetas, eps1, w1, eps2, w2):
    """Feeds a theta_95 sequence through the dual-phase schedule; returns the phase after
    every step (1, 2; 3 = converged)."""
    st = np.array([1, 0], dtype=np.int32)
    out = []
    for t in thetas:
        out.append(int(_load().oracle_converge_update(_p(st), float(t), eps1, int(w1), eps2, int(w2))))
    return out


def viewgraph(W, H, K, T, depths, stride: int = 4, tau: float = 3.0) -> np.ndarray:
    """Round-trip-consistent fraction f[i, j] of view i's grid pixels (Section 3, Viewgraph
    Estimation): n x n, zero diagonal.  depths: per-view (H, W) float maps."""
    n = len(W)
    Wa = np.ascontiguousarray(W, dtype=np.int32)
    Ha = np.ascontiguousarray(H, dtype=np.int32)
    Ka = np.ascontiguousarray(K, dtype=np.float64).reshape(n, 4)
    Ta = np.ascontiguousarray(T, dtype=np.float64).reshape(n, 12)
    Z = np.ascontiguousarray(np.concatenate([np.asarray(d, np.float32).ravel() for d in depths]))
    f = np.zeros((n, n))
    rc = _load().oracle_viewgraph(n, _p(Wa), _p(Ha), _p(Ka), _p(Ta), _p(Z), stride, tau, _p(f))
    if rc:
        raise ValueError(f"oracle_viewgraph failed ({rc})")
    return f


def viewgraph_pairs(frac: np.ndarray, min_frac: float = 0.125) -> np.ndarray:
    """Directed pairs (i, j) of the undirected pairs whose round-trip fraction is at least
    min_frac in both directions, in row-major order."""
    keep = np.minimum(frac, frac.T) >= min_frac
    np.fill_diagonal(keep, False)
    return np.argwhere(keep).astype(np.int32)


def set_threads(n: int = 0) -> int:
    """Threads of the OpenMP loops (n > 0 sets them); returns the count in effect."""
    return int(_load().oracle_set_threads(int(n)))


def lambda_at(step: int, lambda0=10.0, lambda1=6.0, lambda_steps=1000) -> float:
    opt = _Opt(lambda0, lambda1, lambda_steps, 1.0, 1e-6, 0, 0, 0, 0.9, 0.999, 1e-12)
    return float(_load().oracle_lambda(ctypes.byref(opt), step))


def scene_from_synth(sc, maps, rec=None) -> OracleScene:
    """Oracle scene from a ``synth.Scene`` and per-view maps (values the GPU stores)."""
    r = sc.rec if rec is None else rec
    return OracleScene(sc.W, sc.H, sc.K, sc.rec_off, r, maps, sc.pairs)
