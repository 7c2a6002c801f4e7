"""Confocal f-k migration in float64 (test infrastructure only).

Follows Sec. 3.1 (Eq. 2: f = |Psi(x, y, z, t=0)|^2) and the prior-work
pipeline of Alg. 1, step by step, with these readings of the paper:

  * Scaling: each time bin t is multiplied by t / (n - 1) (Alg. 1 builds it
    as linspace(0, 1, n); Sec. 4.2 calls it the normalised time index).
  * Padding: data sits top-left in a (pf*a) x (pf*b) x (pf*n) zero box
    (pf = 2 is the padded configuration; pf = 1 is the unpadded one).
  * The fftshift / ifftshift pair of Alg. 1 only centres the spectrum on the
    signed frequency grid mgrid[-N:N]/N; here the spectrum stays in DFT order
    and signed indices are used directly, so no shift is applied to the data
    and the output is cropped from the top-left corner.
  * Stolt: for the signed indices (p~, q~, m~) with X = p~/(Px/2),
    Y = q~/(Py/2), Z = m~/(Pt/2), the source coordinate along the
    temporal-frequency axis is mu = (Pt/2) * sqrt(s_x^2 X^2 + s_y^2 Y^2 + Z^2)
    with s_x = c dt / (2 dx), s_y = c dt / (2 dy). For a square wall this
    equals Alg. 1's s = N_x d_max / (4 N_z apt/2) with d_max = n c dt.
  * interpn fills 0 outside the sampled range [0, Pt/2 - 1] and the value at
    mu = Pt/2 - 1 exactly is kept; linear interpolation between the two
    neighbouring samples along the contiguous axis (Sec. 4.2 / Listing 2).
  * Only Z > 0 is kept and it is weighted by |Z| / Z' elementwise (Alg. 1's
    |Z_w| / max(Z_w'), read as Listing 2's fabs(fz) * rcp(sqrt_term)).
  * Output: |Psi|^2 on the unpadded top-left [0, a) x [0, b) x [0, n) volume;
    depth index k corresponds to k * c * dt / 2.

Parity: pinned (tests/test_oracle_fk.py): closed-form impulse response for a
zero lateral factor, focusing at the physical lateral factor, point-reflector
peak positions on square and non-square walls, agreement with brute-force
backprojection peaks, and agreement with a non-uniform (interpolation-free)
evaluation of the same Fourier integral.
"""
from __future__ import annotations

import os

import numpy as np
from scipy import fft as sfft

C_LIGHT = 299_792_458.0


def _workers(workers):
    return os.cpu_count() if workers is None else workers


def lateral_factors(bin_width_s: float, wall_w_m: float, wall_h_m: float, nx: int, ny: int,
                    c: float = C_LIGHT):
    """(s_x, s_y) = (c dt / (2 dx), c dt / (2 dy)) with dx = W_x / nx (Alg. 1's s)."""
    dx = wall_w_m / nx
    dy = wall_h_m / ny
    return c * bin_width_s / (2.0 * dx), c * bin_width_s / (2.0 * dy)


def signed_index(N: int) -> np.ndarray:
    """DFT-order signed indices of an N-point axis: 0..N/2-1, -N/2..-1."""
    k = np.arange(N)
    return np.where(k < N // 2, k, k - N)


def padded_length(N: int, pad_factor: int) -> int:
    """Transform length of an axis of N samples: pad_factor 2 zero-pads to the
    smallest power of two >= 2N (exactly 2N for power-of-two N, as in Alg. 1);
    pad_factor 1 keeps N."""
    if pad_factor == 1:
        return N
    L = 1
    while L < pad_factor * N:
        L *= 2
    return L


def fk_spectrum(H: np.ndarray, pad_factor: int = 2, workers=None) -> np.ndarray:
    """Steps (i)-(ii): time scaling t/(n-1), zero padding, forward 3D DFT."""
    H = np.asarray(H, dtype=np.float64)
    a, b, n = H.shape
    ramp = np.arange(n, dtype=np.float64) / (n - 1)
    psi = np.zeros((padded_length(a, pad_factor), padded_length(b, pad_factor), padded_length(n, pad_factor)))
    psi[:a, :b, :n] = H * ramp[None, None, :]
    return sfft.fftn(psi, workers=_workers(workers))


def stolt(U: np.ndarray, s_x: float, s_y: float) -> np.ndarray:
    """Step (iii): Stolt resampling with the Jacobian weight and the Z > 0 mask.

    The grids are those of the padded spectrum (Lx, Ly, Lt): X = p~/(Lx/2),
    Y = q~/(Ly/2), Z = m~/(Lt/2), so the source index is
    mu = sqrt((Lt s_x p~/Lx)^2 + (Lt s_y q~/Ly)^2 + m~^2): the same physical
    Stolt map for any padding (Alg. 1's X = p~/a etc. when L = 2 x size)."""
    Px, Py, Pt = U.shape
    hx, hy, ht = Px // 2, Py // 2, Pt // 2
    X = signed_index(Px) / hx
    Y = signed_index(Py) / hy
    m = np.arange(1, ht)                       # m~ >= 1 (Z > 0); mu >= m~
    Z = m / ht
    Zp = np.sqrt((s_x * X)[:, None, None] ** 2 + (s_y * Y)[None, :, None] ** 2
                 + Z[None, None, :] ** 2)
    mu = ht * Zp
    valid = mu <= ht - 1
    k0 = np.floor(mu).astype(np.int64)
    alpha = mu - k0
    k1 = np.minimum(k0 + 1, ht - 1)
    k0 = np.where(valid, k0, 0)
    k1 = np.where(valid, k1, 0)
    Upos = U[:, :, :ht]
    U0 = np.take_along_axis(Upos, k0, axis=2)
    U1 = np.take_along_axis(Upos, k1, axis=2)
    Vpos = ((1.0 - alpha) * U0 + alpha * U1) * (Z[None, None, :] / Zp)
    Vpos = np.where(valid, Vpos, 0.0)
    V = np.zeros_like(U)
    V[:, :, 1:ht] = Vpos
    return V


def fk_reconstruct(H: np.ndarray, bin_width_s: float, wall_w_m: float, wall_h_m: float, *,
                   pad_factor: int = 2, c: float = C_LIGHT, workers=None,
                   lateral=None, return_complex: bool = False) -> np.ndarray:
    """Confocal f-k migration of a transient H[x][y][t] (Eq. 2, Alg. 1).

    Returns |Psi|^2 as float64 [a][b][n] (or the complex Psi if
    return_complex). `lateral` overrides (s_x, s_y) for tests.
    """
    H = np.asarray(H, dtype=np.float64)
    a, b, n = H.shape
    s_x, s_y = lateral if lateral is not None else lateral_factors(bin_width_s, wall_w_m,
                                                                   wall_h_m, a, b, c)
    U = fk_spectrum(H, pad_factor, workers)
    V = stolt(U, s_x, s_y)
    del U
    psi = sfft.ifftn(V, workers=_workers(workers))[:a, :b, :n]
    if return_complex:
        return psi
    return np.abs(psi) ** 2
