"""Direct spatial Rayleigh-Sommerfeld summation in float64 (test infrastructure only).

Evaluates the phasor-field propagation of Eq. 3 / Eq. 4 without any Fourier
transform or radial approximation: for every wall-grid voxel x_v and depth d,

    I(x_v, d) = sum_f w(f) e^{i kappa_f (sigma_t d + Delta)}
                sum_s P_f(x_s) e^{i sigma_s kappa_f sqrt(|x_v - x_s|^2 + d^2)}.

The radial operator approximates this by construction (Sec. 4.3 explains why
it cannot match it pointwise), so it is used only to pin peak positions.

Parity: pinned (tests/test_oracle_pf.py) by point-reflector focusing.
"""
from __future__ import annotations

import numpy as np

C_LIGHT = 299_792_458.0


def rsd_direct(P: np.ndarray, freqs: np.ndarray, weights: np.ndarray, depths: np.ndarray,
               wall_w_m: float, wall_h_m: float, sigma_s: int = 2, sigma_t: int = 0,
               delta_m: float = 0.0, c: float = C_LIGHT) -> np.ndarray:
    """P[x][y][f] phasors at the wall -> complex I[x][y][d]."""
    a, b, F = P.shape
    xs = -wall_w_m / 2 + (np.arange(a) + 0.5) * (wall_w_m / a)
    ys = -wall_h_m / 2 + (np.arange(b) + 0.5) * (wall_h_m / b)
    wx, wy = np.meshgrid(xs, ys, indexing="ij")
    wx = wx.reshape(-1)
    wy = wy.reshape(-1)
    lat2 = (wx[:, None] - wx[None, :]) ** 2 + (wy[:, None] - wy[None, :]) ** 2   # [v, s]
    kappa = 2.0 * np.pi * np.asarray(freqs) / c
    Pf = P.reshape(a * b, F)
    out = np.zeros((a * b, len(depths)), dtype=np.complex128)
    for di, d in enumerate(depths):
        R = np.sqrt(lat2 + d * d)
        acc = np.zeros(a * b, dtype=np.complex128)
        for fi in range(F):
            ph = np.exp(1j * sigma_s * kappa[fi] * R)                   # [v, s]
            acc += weights[fi] * np.exp(1j * kappa[fi] * (sigma_t * d + delta_m)) * (ph @ Pf[:, fi])
        out[:, di] = acc
    return out.reshape(a, b, len(depths))


def rsd_direct_at(P: np.ndarray, freqs: np.ndarray, weights: np.ndarray, voxels, wall_w_m: float,
                  wall_h_m: float, sigma_s: int = 2, sigma_t: int = 0, delta_m: float = 0.0,
                  c: float = C_LIGHT) -> np.ndarray:
    """The same sum as rsd_direct at chosen voxels only: voxels = [(ix, iy, depth_m), ...]."""
    a, b, F = P.shape
    xs = -wall_w_m / 2 + (np.arange(a) + 0.5) * (wall_w_m / a)
    ys = -wall_h_m / 2 + (np.arange(b) + 0.5) * (wall_h_m / b)
    wx, wy = np.meshgrid(xs, ys, indexing="ij")
    Pf = P.reshape(a * b, F)
    kappa = 2.0 * np.pi * np.asarray(freqs) / c
    out = np.zeros(len(voxels), dtype=np.complex128)
    for n, (ix, iy, d) in enumerate(voxels):
        R = np.sqrt((wx.reshape(-1) - xs[ix]) ** 2 + (wy.reshape(-1) - ys[iy]) ** 2 + d * d)   # [s]
        ph = np.exp(1j * sigma_s * np.outer(R, kappa))                                       # [s, f]
        out[n] = np.sum(weights * np.exp(1j * kappa * (sigma_t * d + delta_m)) * np.sum(ph * Pf, axis=0))
    return out
