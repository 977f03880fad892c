"""Shared test helpers: oracle-built maps, reduced-precision roundings, GPU scene wrappers,
pose-error metrics.  Test infrastructure only."""
from __future__ import annotations

import math

import numpy as np


def oracle_maps_f32(sc):
    """DTF of every view from the oracle's exact EDT, rounded to float32 (what the GPU stores).
    oracle.edt is a C call that releases the GIL, so the views run on a thread per host core."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    with ThreadPoolExecutor() as ex:
        return list(ex.map(lambda e: oracle.edt(e).astype(np.float32), sc.edges))


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16 bits, round to nearest even (finite inputs)."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b >> 16) & 1) + 0x7FFF
    return ((b + r) >> 16).astype(np.uint16)


def bf16_to_f32(bits: np.ndarray) -> np.ndarray:
    return (bits.astype(np.uint32) << 16).view(np.float32)


def scene_part(sc, maps, rec=None, fixed=True):
    return dict(W=sc.W, H=sc.H, K=sc.K, rec_off=sc.rec_off, rec=sc.rec if rec is None else rec,
                maps=maps, pairs=sc.pairs, fixed=sc.fixed if fixed else None)


def gpu_scene(sc, maps, rec=None, record_dtype=0, map_dtype=0, **opt):
    import paper_2607_00579_gb300 as epo
    o = epo.default_options(**opt)
    return epo.Scene([scene_part(sc, maps, rec)], record_dtype=record_dtype, map_dtype=map_dtype, options=o)


def rot_err_deg(A, B):
    out = []
    for a, b in zip(np.asarray(A).reshape(-1, 12), np.asarray(B).reshape(-1, 12)):
        Ra, Rb = a.reshape(3, 4)[:, :3], b.reshape(3, 4)[:, :3]
        c = (np.trace(Ra @ Rb.T) - 1) / 2
        out.append(math.degrees(math.acos(max(-1.0, min(1.0, c)))))
    return np.array(out)


def centres(T):
    M = np.asarray(T).reshape(-1, 3, 4)
    return -np.einsum("nji,nj->ni", M[:, :, :3], M[:, :, 3])


def trans_err(A, B, scale):
    return np.linalg.norm(centres(A) - centres(B), axis=1) / scale


def grad_rel_err(g, ref):
    """max over poses of ||g_i - ref_i|| / max_i ||ref_i|| (6-vector 2-norms)."""
    g = np.asarray(g).reshape(-1, 6)
    ref = np.asarray(ref).reshape(-1, 6)
    return float(np.linalg.norm(g - ref, axis=1).max() / max(np.linalg.norm(ref, axis=1).max(), 1e-300))


def view_subset(sc, maps, views):
    """The scene restricted to `views` (sorted view ids): their records and maps, and the
    pairs with both ends among them, renumbered.  The first kept view is fixed."""
    import synth
    views = np.asarray(sorted(views), dtype=np.int64)
    new_id = -np.ones(sc.n_views, dtype=np.int64)
    new_id[views] = np.arange(len(views))
    keep = (new_id[sc.pairs[:, 0]] >= 0) & (new_id[sc.pairs[:, 1]] >= 0)
    pairs = new_id[sc.pairs[keep]].astype(np.int32)
    recs, gts, offs = [], [], [0]
    for v in views:
        a, b = sc.rec_off[v], sc.rec_off[v + 1]
        recs.append(sc.rec[a:b])
        gts.append(sc.depth_gt_at_rec[a:b])
        offs.append(offs[-1] + (b - a))
    fixed = np.zeros(len(views), dtype=np.uint8)
    fixed[0] = 1
    T_init = sc.T_init[views].copy()
    T_init[0] = sc.T_gt[views[0]]
    sub = synth.Scene(W=sc.W[views], H=sc.H[views], K=sc.K[views], T_gt=sc.T_gt[views], T_init=T_init,
                      rec_off=np.array(offs, dtype=np.int64), rec=np.concatenate(recs, axis=0),
                      edges=[sc.edges[v] for v in views], pairs=pairs, fixed=fixed,
                      scale=synth.scene_scale(sc.T_gt[views]), depth_gt_at_rec=np.concatenate(gts))
    return sub, [maps[v] for v in views]
