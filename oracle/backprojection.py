"""Brute-force confocal backprojection in float64 (test infrastructure only).

A comparison baseline named in Sec. 2: every voxel sums the transient samples
whose round-trip time matches its distance to each wall point. Used only to
pin the peak locations of the f-k oracle on tiny grids.

Voxel (i, j, k) sits below wall sample (i, j) at depth (k + 1/2) c dt / 2, the
centre of time bin k; wall samples are cell centres.

Parity: pinned (tests/test_oracle_fk.py) by peak positions of rendered point
reflectors.
"""
from __future__ import annotations

import numpy as np

C_LIGHT = 299_792_458.0


def backproject(H: np.ndarray, bin_width_s: float, wall_w_m: float, wall_h_m: float,
                c: float = C_LIGHT) -> np.ndarray:
    H = np.asarray(H, dtype=np.float64)
    a, b, n = H.shape
    xs = -wall_w_m / 2 + (np.arange(a) + 0.5) * (wall_w_m / a)
    ys = -wall_h_m / 2 + (np.arange(b) + 0.5) * (wall_h_m / b)
    zs = (np.arange(n) + 0.5) * (c * bin_width_s / 2.0)
    out = np.zeros((a, b, n))
    Hf = H.reshape(a * b, n)
    wx, wy = np.meshgrid(xs, ys, indexing="ij")
    wx = wx.reshape(-1)
    wy = wy.reshape(-1)
    for i in range(a):
        for j in range(b):
            lat2 = (wx - xs[i]) ** 2 + (wy - ys[j]) ** 2                 # [a*b]
            r = np.sqrt(lat2[:, None] + zs[None, :] ** 2)                # [a*b, n]
            t = np.floor(2.0 * r / (c * bin_width_s)).astype(np.int64)
            ok = t < n
            vals = np.where(ok, Hf[np.arange(a * b)[:, None], np.minimum(t, n - 1)], 0.0)
            out[i, j, :] = vals.sum(axis=0)
    return out
