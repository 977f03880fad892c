"""Literal brute-force enumeration of the EPO loss -- TEST INFRASTRUCTURE ONLY.

A second, deliberately naive statement of Eqs. 6-8 in pure Python loops for tiny
scenes.  It shares no helper with ``epo_oracle.c``: each edge pixel p of view i is
lifted with the paper's world-space form X = P_i^-1 K_i^-1 [u, v, 1]^T z (Algorithm 2,
UnprojectEdgesTo3D; the 4x4 inverse is taken with numpy), projected with
pi = K_j P_j X (Eq. 8), the distance transform is bilinearly sampled, clamped at
lambda and passed through the Huber penalty (Eq. 7); per-direction means and the
pair average follow Eq. 6 (Algorithm 3's sum(valid) normaliser by default).

Only the loss is computed here; its gradient is pinned by finite differences of this
function and by the closed forms in the test-suite.
"""
from __future__ import annotations

import math

import numpy as np


def _pose4(T12):
    M = np.eye(4)
    M[:3, :] = np.asarray(T12, dtype=np.float64).reshape(3, 4)
    return M


def brute_loss(W, H, K, rec_off, rec, maps, pairs, T, lam, delta=1.0, eps_z=1e-6, norm_all=False):
    n = len(W)
    Pinv = [np.linalg.inv(_pose4(T[v])) for v in range(n)]
    total = 0.0
    for (i, j) in pairs:
        i, j = int(i), int(j)
        fx_i, fy_i, cx_i, cy_i = K[i]
        fx_j, fy_j, cx_j, cy_j = K[j]
        Pj = _pose4(T[j])
        M = maps[j]
        Wj, Hj = int(W[j]), int(H[j])
        s, cnt = 0.0, 0
        recs = rec[rec_off[i]:rec_off[i + 1]]
        for r in recs:
            u, v, z = float(r[0]), float(r[1]), float(r[2])
            # K_i^-1 [u, v, 1] z, then P_i^-1
            Xc = np.array([(u - cx_i) / fx_i * z, (v - cy_i) / fy_i * z, z, 1.0])
            Xw = Pinv[i] @ Xc
            Y = Pj @ Xw
            if not (Y[2] > eps_z):
                continue
            up = fx_j * Y[0] / Y[2] + cx_j
            vp = fy_j * Y[1] / Y[2] + cy_j
            if not (0.0 <= up <= Wj - 1 and 0.0 <= vp <= Hj - 1):
                continue
            x0 = min(int(math.floor(up)), Wj - 2)
            y0 = min(int(math.floor(vp)), Hj - 2)
            a, b = up - x0, vp - y0
            d = ((1 - a) * (1 - b) * M[y0][x0] + a * (1 - b) * M[y0][x0 + 1]
                 + (1 - a) * b * M[y0 + 1][x0] + a * b * M[y0 + 1][x0 + 1])
            dh = min(d, lam)
            rho = 0.5 * dh * dh if abs(dh) <= delta else delta * (abs(dh) - 0.5 * delta)
            s += rho
            cnt += 1
        denom = len(recs) if norm_all else cnt
        total += s / denom if denom > 0 else 0.0
    return 2.0 * total / len(pairs) if len(pairs) else 0.0
