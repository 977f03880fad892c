"""GB300-native EPO edge-alignment library (Python side).

``_binding`` exposes the C ABI of ``include/epo.h`` under the same names.  This module
adds convenience wrappers: ``Scene`` (one handle over one or many scenes, numpy or torch
inputs), ``EdgeLoss`` (a ``torch.autograd.Function`` whose forward and backward are the
library's forward and recomputing adjoint kernels) and GPU distance-field construction.
PyTorch is used for device memory and streams only; every step of the objective runs in
the library's CUDA kernels and the import fails loudly when the library cannot load.
"""
from __future__ import annotations

import ctypes
from typing import List, Optional, Sequence

import numpy as np

from . import _binding as B
from ._binding import (EPO_BF16, EPO_F16, EPO_F32, EPO_GATHER_AUTO, EPO_GATHER_LDG, EPO_GATHER_MIX, EPO_GATHER_TEX,
                       EPO_NORM_ALL, EPO_NORM_VALID, EpoError, default_options)

__all__ = ["Scene", "EdgeLoss", "distance_field", "round_bf16", "default_options", "EpoError",
           "EPO_F32", "EPO_F16", "EPO_BF16", "EPO_NORM_VALID", "EPO_NORM_ALL", "EPO_GATHER_AUTO",
           "EPO_GATHER_LDG", "EPO_GATHER_TEX", "EPO_GATHER_MIX", "library_path"]


def library_path() -> str:
    import os
    return os.environ.get("EPO_LIBRARY") or B.LIB_PATH


def _current_stream() -> int:
    import torch
    return torch.cuda.current_stream().cuda_stream


class _SceneData:
    """Keeps the marshalled descriptor arrays alive while the library copies them."""

    def __init__(self, W, H, K, rec_off, rec, maps, pairs, fixed, record_dtype, map_dtype, on_device):
        n = len(W)
        self.views = (B.epo_view_desc * n)()
        self.keep = []
        rec_off = np.asarray(rec_off, dtype=np.int64)
        for v in range(n):
            d = self.views[v]
            d.W, d.H = int(W[v]), int(H[v])
            d.fx, d.fy, d.cx, d.cy = (float(x) for x in K[v])
            lo, hi = int(rec_off[v]), int(rec_off[v + 1])
            if on_device:
                r = rec[lo:hi]
                d.records = r.data_ptr() if hi > lo else None
                d.map = maps[v].data_ptr()
                self.keep += [r, maps[v]]
            else:
                r = np.ascontiguousarray(rec[lo:hi])
                m = np.ascontiguousarray(maps[v])
                d.records = r.ctypes.data if hi > lo else None
                d.map = m.ctypes.data
                self.keep += [r, m]
            d.n_records = hi - lo
        self.pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1)
        self.fixed = None if fixed is None else np.ascontiguousarray(fixed, dtype=np.uint8)
        self.desc = B.epo_scene_desc()
        self.desc.n_views = n
        self.desc.views = ctypes.cast(self.views, ctypes.POINTER(B.epo_view_desc))
        self.desc.n_pairs = self.pairs.size // 2
        self.desc.pairs = self.pairs.ctypes.data
        self.desc.fixed = None if self.fixed is None else self.fixed.ctypes.data
        self.desc.record_dtype = record_dtype
        self.desc.map_dtype = map_dtype
        self.desc.pointers_on_device = 1 if on_device else 0


class Scene:
    """One library handle over one scene or a batch of scenes.

    ``parts``: list of dicts with keys W, H, K (n,4), rec_off (n+1), rec ((n_rec,4) f32 records
    or (n_rec,4) uint16 packed FP16-depth records), maps (list of (H,W) f32 or uint16 bf16
    bits), pairs (P,2), fixed (n,) -- numpy (host) or torch CUDA tensors (device).
    """

    def __init__(self, parts: Sequence[dict], record_dtype: int = EPO_F32, map_dtype: int = EPO_F32,
                 options: Optional[B.epo_options] = None, stream: Optional[int] = None,
                 on_device: bool = False):
        self._stream = _current_stream() if stream is None else stream
        datas = [_SceneData(p["W"], p["H"], p["K"], p["rec_off"], p["rec"], p["maps"], p["pairs"],
                            p.get("fixed"), record_dtype, map_dtype, on_device) for p in parts]
        opts = options if options is not None else default_options()
        self.handle = B.epo_create_batch([d.desc for d in datas], opts, self._stream)
        info = B.epo_scene_info_get(self.handle)
        self.n_scenes, self.n_views, self.n_pairs = info.n_scenes, info.n_views, info.n_pairs

    @classmethod
    def single(cls, W, H, K, rec_off, rec, maps, pairs, fixed=None, **kw) -> "Scene":
        return cls([dict(W=W, H=H, K=K, rec_off=rec_off, rec=rec, maps=maps, pairs=pairs, fixed=fixed)], **kw)

    def close(self):
        if getattr(self, "handle", None):
            B.epo_destroy_scene(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- state ----
    def info(self) -> B.epo_scene_info:
        return B.epo_scene_info_get(self.handle)

    def set_poses(self, T: np.ndarray):
        B.epo_set_poses(self.handle, np.ascontiguousarray(T, dtype=np.float64).reshape(self.n_views, 12))

    def get_poses(self) -> np.ndarray:
        T = np.zeros((self.n_views, 12))
        B.epo_get_poses(self.handle, T)
        return T

    def get_state(self):
        step = np.zeros(1, dtype=np.int64)
        m = np.zeros((self.n_views, 6))
        v = np.zeros((self.n_views, 6))
        B.epo_get_state(self.handle, step, m, v)
        return int(step[0]), m, v

    def set_state(self, step: int, m=None, v=None):
        m = None if m is None else np.ascontiguousarray(m, dtype=np.float64)
        v = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
        B.epo_set_state(self.handle, int(step), m, v)

    # ---- evaluation ----
    def loss_and_grad(self):
        loss = np.zeros(self.n_scenes)
        grad = np.zeros((self.n_views, 6))
        B.epo_loss_and_grad(self.handle, loss, grad)
        return loss, grad

    def pair_stats(self) -> np.ndarray:
        st = np.zeros((self.n_pairs, 8))
        B.epo_pair_stats(self.handle, st)
        return st

    def step(self, n: int = 1):
        B.epo_step(self.handle, n)

    def step_async(self, n: int = 1):
        B.epo_step_async(self.handle, n)

    def step_plain(self, n: int = 1):
        B.epo_step_plain(self.handle, n)

    def check(self):
        B.epo_check(self.handle)

    def autotune(self):
        B.epo_autotune(self.handle)

    def set_pair_subset(self, ids):
        B.epo_set_pair_subset(self.handle, ids)


class EdgeLoss:
    """``torch.autograd.Function`` over the twists xi (n_views x 6, float64, CUDA):
    loss(xi) = L(Exp(xi_i) T_i) per scene.  Forward = the library's forward kernel;
    backward = its recomputing adjoint kernel followed by J_l(xi)^T."""

    _fn = None

    @classmethod
    def apply(cls, xi, scene: Scene):
        if cls._fn is None:
            import torch

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, x, sc):
                    x = x.contiguous()
                    loss = torch.empty(sc.n_scenes, dtype=torch.float64, device=x.device)
                    B.epo_forward_dev(sc.handle, x, loss)
                    ctx.save_for_backward(x)
                    ctx.scene = sc
                    return loss

                @staticmethod
                def backward(ctx, gloss):
                    (x,) = ctx.saved_tensors
                    g = torch.empty_like(x)
                    B.epo_backward_dev(ctx.scene.handle, x, gloss.contiguous().to(torch.float64), g)
                    return g, None

            cls._fn = _F
        return cls._fn.apply(xi, scene)


def distance_field(edges, stream: Optional[int] = None):
    """Exact distance transform field of a (H, W) uint8 CUDA tensor -> (H, W) float32 CUDA tensor."""
    import torch
    e = edges.contiguous()
    H, W = e.shape
    out = torch.empty((H, W), dtype=torch.float32, device=e.device)
    B.epo_distance_field(e, W, H, out, _current_stream() if stream is None else stream)
    return out


def build_viewgraph(W, H, K, T, depths, stride: int = 4, tau: float = 3.0, min_frac: float = 0.125,
                    stream: Optional[int] = None):
    """Viewgraph estimation on the GPU (Section 3): returns (frac (n, n), pairs (m, 2)) for
    per-view depth maps given as CUDA float tensors (H, W) or one concatenated tensor."""
    import torch
    if isinstance(depths, (list, tuple)):
        depths = torch.cat([d.reshape(-1).float() for d in depths])
    depths = depths.contiguous()
    return B.epo_build_viewgraph(W, H, K, T, depths, stride, tau, min_frac,
                                 _current_stream() if stream is None else stream)


def round_bf16(x, stream: Optional[int] = None):
    """float32 CUDA tensor -> the bfloat16 bits (int16 tensor of the same shape), RNE."""
    import torch
    x = x.contiguous()
    out = torch.empty(x.shape, dtype=torch.int16, device=x.device)
    B.epo_round_bf16(x, out, x.numel(), _current_stream() if stream is None else stream)
    return out
