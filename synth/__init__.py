"""Seeded synthetic scenes shaped like EPO's workloads (input generation only).

The paper measures on real image collections (ScanNet++, TerraSky3D, Mip-NeRF 360)
with VGGT predictions (Section 4).  None of those are available, so every test and
benchmark input is generated here from a seed: a world of random rectangles and
3D line segments, cameras on a ring or a random walk around it, ray-cast depth
(optionally multiplied by a smooth low-frequency noise field to mimic a
feed-forward depth prediction), edge pixels = visible segment pixels plus the
foreground side of depth discontinuities, uniformly sub-sampled to a target count
per view (the E_max sub-sampling of Algorithm 1), k-nearest-neighbour directed
view pairs, and ground-truth poses perturbed by Gaussian rotation/translation
noise.

This module is shared by the oracle side and the CUDA side strictly as a source
of inputs.  It contains no part of the alignment objective: no distance
transform, no relative-pose projection of edge records, no robust penalty, no
gradient.  The distance maps are built from the returned edge masks by the
caller (the CPU oracle in tests, the library's own distance-field kernel in the
benchmark).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "scenegen.c")
_LIB_PATH = os.path.join(_HERE, "_scenegen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the rasteriser with gcc (OpenMP, no arch-specific flags)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        lib.synth_render_views.argtypes = [P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int, P, P, P, P,
                                           ctypes.c_double, P, P, P, P]
        lib.synth_render_views.restype = ctypes.c_int64
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


# --------------------------------------------------------------------------------------
# workload presets (named by what they are)
# --------------------------------------------------------------------------------------
@dataclasses.dataclass
class SceneSpec:
    n_views: int
    width: int
    height: int
    n_planes: int
    n_segments: int
    edges_per_view: Optional[int] = None      # target count per view ...
    edge_density: Optional[float] = None      # ... or a fraction of the pixels
    knn: Optional[int] = None                 # None = all ordered pairs
    trajectory: str = "ring"                  # "ring" | "walk"
    focal: Optional[float] = None             # None = 1.1 * width
    depth_noise: float = 0.0                  # sigma of the multiplicative depth field
    rot_noise_deg: float = 1.0
    trans_noise_frac: float = 0.02
    seed: int = 20260000
    cube: float = 10.0
    ring_radius: float = 15.0


RING8_128x96 = SceneSpec(n_views=8, width=128, height=96, n_planes=12, n_segments=40,
                         edges_per_view=2000, knn=None, focal=100.0, depth_noise=0.0,
                         rot_noise_deg=1.0, trans_noise_frac=0.02, seed=20260001)
RING32_518x392 = SceneSpec(n_views=32, width=518, height=392, n_planes=24, n_segments=160,
                           edges_per_view=20000, knn=8, depth_noise=0.03,
                           rot_noise_deg=2.0, trans_noise_frac=0.05, seed=20260002)
WALK200_518x392 = SceneSpec(n_views=200, width=518, height=392, n_planes=60, n_segments=400,
                            edges_per_view=30000, knn=10, trajectory="walk", depth_noise=0.03,
                            rot_noise_deg=2.0, trans_noise_frac=0.05, seed=20260003)
RING500_518x518 = SceneSpec(n_views=500, width=518, height=518, n_planes=60, n_segments=400,
                            edges_per_view=40000, knn=12, depth_noise=0.03,
                            rot_noise_deg=2.0, trans_noise_frac=0.05, seed=20260005)


def batch64_uneven_specs(n_scenes: int = 64, seed: int = 20260004) -> List[SceneSpec]:
    """64 independent scenes: views U[8,120], resolution from {256x192, 518x392, 518x518},
    k = 8, edge density U[2%, 8%] of the pixels."""
    rng = np.random.default_rng(seed)
    res = [(256, 192), (518, 392), (518, 518)]
    specs = []
    for s in range(n_scenes):
        n = int(rng.integers(8, 121))
        w, h = res[int(rng.integers(0, 3))]
        dens = float(rng.uniform(0.02, 0.08))
        specs.append(SceneSpec(n_views=n, width=w, height=h, n_planes=24, n_segments=150,
                               edge_density=dens, knn=8, depth_noise=0.03, rot_noise_deg=2.0,
                               trans_noise_frac=0.05, seed=seed * 1000 + s))
    return specs


# --------------------------------------------------------------------------------------
# geometry helpers (input generation only)
# --------------------------------------------------------------------------------------
def _look_at(C: np.ndarray, target: np.ndarray) -> np.ndarray:
    """World->camera [R|t] (x right, y down, z forward) for a camera at C looking at target."""
    f = target - C
    f = f / np.linalg.norm(f)
    up = np.array([0.0, 0.0, 1.0])
    r = np.cross(f, up)
    r = r / np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    t = -R @ C
    return np.concatenate([R, t[:, None]], axis=1)


def _rotvec_to_matrix(w: np.ndarray) -> np.ndarray:
    from scipy.spatial.transform import Rotation
    return Rotation.from_rotvec(w).as_matrix()


def _world(spec: SceneSpec, rng: np.random.Generator):
    half = spec.cube / 2
    planes = np.zeros((spec.n_planes, 15))
    for p in range(spec.n_planes):
        c = rng.uniform(-half, half, 3)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        a = rng.normal(size=3)
        e1 = np.cross(n, a)
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(n, e1)
        s1, s2 = rng.uniform(1.0, 4.0, 2)
        planes[p, 0:3] = c
        planes[p, 3:6] = e1
        planes[p, 6:9] = e2
        planes[p, 9:12] = n
        planes[p, 12] = s1 / 2
        planes[p, 13] = s2 / 2
    segs = rng.uniform(-half, half, (spec.n_segments, 6))
    return planes, segs


def _cameras(spec: SceneSpec, rng: np.random.Generator) -> np.ndarray:
    n = spec.n_views
    T = np.zeros((n, 12))
    if spec.trajectory == "ring":
        for k in range(n):
            th = 2 * np.pi * k / n + rng.normal(0, 0.02)
            C = np.array([spec.ring_radius * np.cos(th), spec.ring_radius * np.sin(th),
                          rng.uniform(-1.0, 1.0)])
            T[k] = _look_at(C, rng.normal(0, 0.2, 3)).reshape(-1)
    elif spec.trajectory == "walk":
        # random walk of step 0.5 around the scene: the heading angle drifts, the
        # radius and height wander inside a band, the camera looks inward.
        th = 0.0
        rad = spec.ring_radius
        hgt = 0.0
        dth = 0.5 / spec.ring_radius
        for k in range(n):
            th += dth * (1.0 + 0.3 * rng.normal())
            rad = float(np.clip(rad + 0.5 * rng.normal() * 0.5, 12.0, 18.0))
            hgt = float(np.clip(hgt + 0.5 * rng.normal() * 0.5, -2.0, 2.0))
            C = np.array([rad * np.cos(th), rad * np.sin(th), hgt])
            T[k] = _look_at(C, rng.normal(0, 1.0, 3)).reshape(-1)
    else:
        raise ValueError(spec.trajectory)
    return T


def _centres(T: np.ndarray) -> np.ndarray:
    R = T.reshape(-1, 3, 4)[:, :, :3]
    t = T.reshape(-1, 3, 4)[:, :, 3]
    return -np.einsum("nji,nj->ni", R, t)


def scene_scale(T: np.ndarray) -> float:
    """RMS distance of the camera centres from their centroid."""
    C = _centres(T)
    return float(np.sqrt(np.mean(np.sum((C - C.mean(0)) ** 2, axis=1))))


def _smooth_noise(rng: np.random.Generator, W: int, H: int, sigma: float) -> np.ndarray:
    """1 + n(x, y): a 4x3 grid of Gaussians, bicubically (Keys, a = -0.5) upsampled, scaled
    to standard deviation sigma over the image."""
    gx, gy = 4, 3
    g = rng.normal(size=(gy, gx))

    def keys(t):
        t = np.abs(t)
        a = -0.5
        return np.where(t <= 1, (a + 2) * t**3 - (a + 3) * t**2 + 1,
                        np.where(t < 2, a * t**3 - 5 * a * t**2 + 8 * a * t - 4 * a, 0.0))

    xs = np.linspace(0, gx - 1, W)
    ys = np.linspace(0, gy - 1, H)

    def interp_matrix(coords, n):
        M = np.zeros((len(coords), n))
        rows = np.arange(len(coords))
        b = np.floor(coords).astype(np.int64)
        for o in range(-1, 3):  # the four taps, accumulated in tap order
            k = b + o
            np.add.at(M, (rows, np.clip(k, 0, n - 1)), keys(coords - k))
        return M

    Mx = interp_matrix(xs, gx)
    My = interp_matrix(ys, gy)
    f = My @ g @ Mx.T
    f = f - f.mean()
    sd = f.std()
    if sd > 0:
        f = f * (sigma / sd)
    return 1.0 + f


@dataclasses.dataclass
class Scene:
    """One synthetic scene.  Arrays are numpy; records are the kernel's FP32 layout."""
    W: np.ndarray            # (n,) int32
    H: np.ndarray            # (n,) int32
    K: np.ndarray            # (n, 4) float64 fx fy cx cy
    T_gt: np.ndarray         # (n, 12) float64, world->camera [R|t] row-major
    T_init: np.ndarray       # (n, 12) float64, perturbed initial poses
    rec_off: np.ndarray      # (n+1,) int64 CSR offsets into rec
    rec: np.ndarray          # (n_rec, 4) float32 {u, v, z, 0}
    edges: List[np.ndarray]  # per view (H, W) uint8, full (pre-sub-sampling) edge mask
    pairs: np.ndarray        # (P, 2) int32 directed (i -> j)
    fixed: np.ndarray        # (n,) uint8
    scale: float             # RMS distance of the GT camera centres from their centroid
    depth_gt_at_rec: np.ndarray  # (n_rec,) float64 noise-free depth of every record
    depth: Optional[List[np.ndarray]] = None  # per view (H, W) rendered GT depth (keep_depth=True)

    @property
    def n_views(self) -> int:
        return int(self.W.shape[0])

    @property
    def n_pairs(self) -> int:
        return int(self.pairs.shape[0])

    def records(self, v: int) -> np.ndarray:
        return self.rec[self.rec_off[v]:self.rec_off[v + 1]]

    def evals(self) -> int:
        """Edge-pixel x pair evaluations per objective evaluation: sum over pairs of |E_i|."""
        cnt = np.diff(self.rec_off)
        return int(cnt[self.pairs[:, 0]].sum())


def _pairs(spec: SceneSpec, T_gt: np.ndarray) -> np.ndarray:
    n = spec.n_views
    if spec.knn is None:
        return np.array([(i, j) for i in range(n) for j in range(n) if i != j], dtype=np.int32)
    C = _centres(T_gt)
    D = np.linalg.norm(C[:, None, :] - C[None, :, :], axis=2)
    out = []
    k = min(spec.knn, n - 1)
    for i in range(n):
        order = np.argsort(D[i], kind="stable")
        nb = [int(j) for j in order if j != i][:k]
        out.extend((i, j) for j in nb)
    return np.array(out, dtype=np.int32)


def make_scene(spec: SceneSpec, keep_depth: bool = False) -> Scene:
    rng = np.random.default_rng(spec.seed)
    planes, segs = _world(spec, rng)
    T_gt = _cameras(spec, rng)
    n = spec.n_views
    W = np.full(n, spec.width, dtype=np.int32)
    H = np.full(n, spec.height, dtype=np.int32)
    f = spec.focal if spec.focal is not None else 1.1 * spec.width
    K = np.zeros((n, 4))
    K[:, 0] = f
    K[:, 1] = f
    K[:, 2] = (spec.width - 1) / 2.0
    K[:, 3] = (spec.height - 1) / 2.0
    px_off = np.zeros(n + 1, dtype=np.int64)
    px_off[1:] = np.cumsum(W.astype(np.int64) * H)
    depth = np.zeros(int(px_off[-1]), dtype=np.float32)
    edge = np.zeros(int(px_off[-1]), dtype=np.uint8)
    ecount = np.zeros(n, dtype=np.int64)
    lib = _load()
    planes_c = np.ascontiguousarray(planes)
    segs_c = np.ascontiguousarray(segs)
    Kc = np.ascontiguousarray(K)
    Tc = np.ascontiguousarray(T_gt)
    rc = lib.synth_render_views(_ptr(planes_c), planes.shape[0], _ptr(segs_c), segs.shape[0], n,
                                _ptr(W), _ptr(H), _ptr(Kc), _ptr(Tc), ctypes.c_double(0.05),
                                _ptr(px_off), _ptr(depth), _ptr(edge), _ptr(ecount))
    if rc != 0:
        raise RuntimeError("synthetic rendering failed")
    recs, gts, offs, edges, depths = [], [], [0], [], []
    for v in range(n):
        w, h = int(W[v]), int(H[v])
        dmap = depth[px_off[v]:px_off[v + 1]].reshape(h, w)
        emap = edge[px_off[v]:px_off[v + 1]].reshape(h, w)
        edges.append(emap.copy())
        if keep_depth:
            depths.append(dmap.copy())
        ys, xs = np.nonzero(emap)           # raster order
        target = spec.edges_per_view
        if spec.edge_density is not None:
            target = int(round(spec.edge_density * w * h))
        if target is not None and len(xs) > target:
            sel = np.sort(rng.choice(len(xs), size=target, replace=False))
            xs, ys = xs[sel], ys[sel]
        zgt = dmap[ys, xs].astype(np.float64)
        if spec.depth_noise > 0:
            field = _smooth_noise(rng, w, h, spec.depth_noise)
            z = zgt * field[ys, xs]
        else:
            z = zgt
        r = np.zeros((len(xs), 4), dtype=np.float32)
        r[:, 0] = xs
        r[:, 1] = ys
        r[:, 2] = z
        recs.append(r)
        gts.append(zgt)
        offs.append(offs[-1] + len(xs))
    # perturbation: left rotation noise, camera-centre noise; view 0 stays at GT
    scale = scene_scale(T_gt)
    T_init = T_gt.copy()
    for v in range(1, n):
        Rg = T_gt[v].reshape(3, 4)[:, :3]
        Cg = _centres(T_gt[v:v + 1])[0]
        dR = _rotvec_to_matrix(rng.normal(0, np.deg2rad(spec.rot_noise_deg), 3))
        R = dR @ Rg
        C = Cg + rng.normal(0, spec.trans_noise_frac * scale, 3)
        T_init[v] = np.concatenate([R, (-R @ C)[:, None]], axis=1).reshape(-1)
    fixed = np.zeros(n, dtype=np.uint8)
    fixed[0] = 1
    return Scene(W=W, H=H, K=K, T_gt=T_gt, T_init=T_init,
                 rec_off=np.array(offs, dtype=np.int64),
                 rec=np.concatenate(recs, axis=0) if recs else np.zeros((0, 4), np.float32),
                 edges=edges, pairs=_pairs(spec, T_gt), fixed=fixed, scale=scale,
                 depth_gt_at_rec=np.concatenate(gts) if gts else np.zeros(0),
                 depth=depths if keep_depth else None)


def records_f16(rec: np.ndarray) -> np.ndarray:
    """Pack FP32 records {u, v, z, 0} into the 8-byte form {u16 u, u16 v, f16 z, u16 0}."""
    out = np.zeros((rec.shape[0], 4), dtype=np.uint16)
    out[:, 0] = rec[:, 0].astype(np.uint16)
    out[:, 1] = rec[:, 1].astype(np.uint16)
    out[:, 2] = rec[:, 2].astype(np.float16).view(np.uint16)
    return out


def records_f16_widened(rec: np.ndarray) -> np.ndarray:
    """The values the 8-byte form stores, widened back to FP32 {u, v, z, 0}."""
    out = rec.copy()
    out[:, 2] = rec[:, 2].astype(np.float16).astype(np.float32)
    return out


def pose_mlp_init(seed: int = 20260100) -> np.ndarray:
    """Initial parameters of the pose MLP (Section 3, Pose Refinement): Kaiming-normal weights
    (std sqrt(2 / fan_in)) for the first five layers, the last layer zero, biases zero.  Flat
    float32 in the layout W1 (128x12), b1, W2..W5 (128x128), b2..b5, W6 (12x128), b6."""
    rng = np.random.default_rng(seed)
    dims = [(128, 12), (128, 128), (128, 128), (128, 128), (128, 128), (12, 128)]
    parts = []
    for l, (o, i) in enumerate(dims):
        W = np.zeros((o, i)) if l == 5 else rng.normal(0.0, np.sqrt(2.0 / i), (o, i))
        parts += [W.ravel(), np.zeros(o)]
    return np.concatenate(parts).astype(np.float32)
