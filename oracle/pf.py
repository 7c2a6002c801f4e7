"""Symmetry-aware phasor-field (RSD) reconstruction in float64 (test infrastructure only).

Follows Sec. 3.1 (phasor fields, Eq. 3), Sec. 4.3 (ring decomposition Eq. 4,
ring basis Eq. 5, radial kernel Eq. 6, propagation sum Eq. 7), the
supplementary radial sampling equations (radial extent, ring count,
trapezoid weights, radial sample count, cutoff, bin coordinate, smoothstep
taper) and Alg. 4, with these readings where the paper is silent:

  * Virtual wave: wavelength lambda = 4 dx unless given; centre frequency
    f0 = c / lambda; bin spacing df = 1 / (Lt dt) with Lt = n for power-of-two
    n and the next power of two otherwise (zero-padded temporal transform);
    centre bin k0 = round(f0/df).
    "cycles" wide means +-3 sigma_t spans `cycles` periods:
    sigma_t = cycles / (6 f0), sigma_f = 1 / (2 pi sigma_t). The band keeps
    bins k0 - K_h .. k0 + K_h with K_h = round(5 sigma_f / df), clipped to
    [1, n/2 - 1]; w(f) = exp(-(f_k - f0)^2 / (2 sigma_f^2)).
  * Phasors: P(x, y, f) = sum_t H(x, y, t) exp(-2 pi i k_f t / Lt), Lt the
    temporal transform length above (forward DFT sign e^{-i}); w(f) is
    applied inside the depth sum (Alg. 4).
  * Spectral coordinates: the top-left padded grid is Nu x Nv = 2a x 2b
    (the next powers of two >= 2a, 2b for other sizes)
    with physical sides Nu dx and Nv dy; DFT index (kx, ky) has signed indices
    (kx~, ky~) and radius rho = sqrt((kx~/(Nu dx))^2 + (ky~/(Nv dy))^2).
  * Kernel phase e^{+i kappa sigma_s sqrt(r^2 + d^2)} (Eq. 4) with
    kappa_f = 2 pi f_k / c; the (sigma_t d + Delta) phase applied after the
    ring sum. No 1/(dx dy) continuous-to-discrete factor is applied.
  * Integer rounding of N_r and N_rho uses ceil(x - 1e-9) so that values that
    are integers in exact arithmetic (2 r_max rho_max = N on square grids) do
    not round up by floating-point noise.
  * rhoCutoffIndex of Listing 3 is floor(rho~_cutoff).
  * Inverse DFT carries 1/(Nu Nv); the volume is |I| on the top-left a x b.
  * Depth planes d_j = d_min + j (d_max - d_min) / (D - 1).

Parity: pinned (tests/test_oracle_pf.py): the supplementary worked example
(190 x 190, N_r = 128, N_rho = 256, rho_max = 70.34, rho_cutoff = 47.02),
J0 against its integral definition and tabulated zeros, the ring basis
against angular quadrature of a unit ring's 2D Fourier transform, the
radial quadrature against the closed-form Hankel transform of a Gaussian,
taper endpoints, the cos/sin linearity identity, single-point focusing,
peak agreement with the direct spatial RSD summation, and the complex field
of propagate against the direct sum with the fixed dx dy area factor (this
pins w(f) and the absolute and per-frequency amplitude of K_r).
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass

import numpy as np
from scipy import fft as sfft
from scipy import special

C_LIGHT = 299_792_458.0
TAPER_BINS = 8.0


def _workers(workers):
    return os.cpu_count() if workers is None else workers


def _ceil_int(x: float) -> int:
    return int(math.ceil(x - 1e-9))


def _pow2_at_least(x: int) -> int:
    return 1 << int(math.ceil(math.log2(x)))


def _padded(N: int, pad_factor: int) -> int:
    """Spatial transform length: the smallest power of two >= pad_factor * N
    (exactly 2N for power-of-two N, Alg. 4's pad_tl)."""
    return _pow2_at_least(pad_factor * N)


def temporal_length(nt: int) -> int:
    """Length of the temporal DFT: nt for power-of-two nt, otherwise the
    transient zero-padded to the next power of two (finer band spacing)."""
    return _pow2_at_least(nt)


@dataclass
class Band:
    f0: float
    df: float
    k0: int
    k_half: int
    bins: np.ndarray        # int [F]
    freqs: np.ndarray       # Hz [F]
    weights: np.ndarray     # w(f) [F]
    sigma_f: float


def virtual_wave_band(nt: int, bin_width_s: float, wavelength_m: float, cycles: float,
                      c: float = C_LIGHT) -> Band:
    """Temporal-frequency band of the Gaussian-windowed virtual wave (Sec. 3.1)."""
    f0 = c / wavelength_m
    df = 1.0 / (nt * bin_width_s)
    k0 = int(round(f0 / df))
    sigma_t = cycles / (6.0 * f0)
    sigma_f = 1.0 / (2.0 * math.pi * sigma_t)
    k_half = int(round(5.0 * sigma_f / df))
    lo = max(1, k0 - k_half)
    hi = min(nt // 2 - 1, k0 + k_half)
    bins = np.arange(lo, hi + 1)
    freqs = bins * df
    w = np.exp(-((freqs - f0) ** 2) / (2.0 * sigma_f ** 2))
    return Band(f0, df, k0, k_half, bins, freqs, w, sigma_f)


@dataclass
class RadialSampling:
    r_max: float
    rho_max: float
    n_r: int
    n_rho: int
    dr: float
    r: np.ndarray
    q: np.ndarray
    rho: np.ndarray
    rho_cut: float
    rho_cut_bin: float
    nyquist_rings: int
    nyquist_rho: int


def radial_sampling(Nu: int, Nv: int, dx: float, dy: float, sigma_s: int,
                    lambda_min: float) -> RadialSampling:
    """Supplementary radial extent, ring count, trapezoid weights, sample count, cutoff."""
    r_max = math.sqrt((0.5 * Nu * dx) ** 2 + (0.5 * Nv * dy) ** 2)
    rho_max = math.sqrt((1.0 / (2.0 * dx)) ** 2 + (1.0 / (2.0 * dy)) ** 2)
    nyq_r = _ceil_int(2.0 * sigma_s * r_max / lambda_min) + 1
    n_r = max(2, _pow2_at_least(nyq_r))
    dr = r_max / (n_r - 1)
    r = np.arange(n_r) * dr
    q = trapezoid_weights(n_r, dr)
    nyq_rho = _ceil_int(2.0 * r_max * rho_max) + 1
    n_rho = _pow2_at_least(nyq_rho)
    rho = np.arange(n_rho) * (rho_max / (n_rho - 1))
    rho_cut = min(rho_max, 0.5 * (n_r - 1) / r_max)
    rho_cut_bin = rho_cut * (n_rho - 1) / rho_max
    return RadialSampling(r_max, rho_max, n_r, n_rho, dr, r, q, rho, rho_cut, rho_cut_bin,
                          nyq_r, nyq_rho)


def trapezoid_weights(n_r: int, dr: float) -> np.ndarray:
    """q_0 = q_{N-1} = dr/2, q_j = dr otherwise."""
    q = np.full(n_r, dr)
    q[0] = q[-1] = 0.5 * dr
    return q


def ring_basis(r: np.ndarray, rho: np.ndarray) -> np.ndarray:
    """B(r, rho) = 2 pi r J0(2 pi r rho) (Eq. 5), shape [len(rho), len(r)]."""
    r = np.asarray(r, dtype=np.float64)
    rho = np.asarray(rho, dtype=np.float64)
    return 2.0 * np.pi * r[None, :] * special.j0(2.0 * np.pi * r[None, :] * rho[:, None])


def ring_integral(A: np.ndarray, r: np.ndarray, q: np.ndarray, rho: np.ndarray) -> np.ndarray:
    """sum_j q_j A(r_j, ...) B(r_j, rho_i) (quadrature of Eq. 6).

    A has shape [N_r, ...]; the result has shape [len(rho), ...].
    """
    B = ring_basis(r, rho) * q[None, :]
    flat = A.reshape(A.shape[0], -1)
    out = (B @ flat.real) + 1j * (B @ flat.imag) if np.iscomplexobj(flat) else B @ flat
    return out.reshape((len(rho),) + A.shape[1:])


def taper(rho_bin: np.ndarray, rho_cut_bin: float, width: float = TAPER_BINS) -> np.ndarray:
    """Smoothstep a_cutoff over the last `width` bins below the cutoff."""
    rb = np.asarray(rho_bin, dtype=np.float64)
    t = (rho_cut_bin - rb) / width
    a = t * t * (3.0 - 2.0 * t)
    a = np.where(rb <= rho_cut_bin - width, 1.0, a)
    a = np.where(rb >= rho_cut_bin, 0.0, a)
    return a


def lerp_indices(rho_bin: np.ndarray, rho_cut_bin: float, n_rho: int):
    """Listing 3's clamped neighbour indices and interpolation weight."""
    rb = np.asarray(rho_bin, dtype=np.float64)
    i_c = int(math.floor(rho_cut_bin))
    last_base = max(0, min(i_c - 1, n_rho - 2))
    i0 = np.clip(np.floor(rb).astype(np.int64), 0, last_base)
    i1 = np.minimum(i0 + 1, i_c)
    alpha = rb - i0
    return i0, i1, alpha


@dataclass
class PhasorPlan:
    nx: int
    ny: int
    nt: int
    bin_width_s: float
    wall_w_m: float
    wall_h_m: float
    pad_factor: int
    dx: float
    dy: float
    Nu: int
    Nv: int
    wavelength_m: float
    cycles: float
    band: Band
    lambda_min: float
    sigma_s: int
    sigma_t: int
    delta_m: float
    depths: np.ndarray
    radial: RadialSampling
    K_r: np.ndarray          # complex128 [N_rho][F][D]


def depth_planes(n_depths: int, d_min: float, d_max: float) -> np.ndarray:
    if n_depths == 1:
        return np.array([d_min])
    return d_min + np.arange(n_depths) * ((d_max - d_min) / (n_depths - 1))


def make_plan(nx: int, ny: int, nt: int, bin_width_s: float, wall_w_m: float, wall_h_m: float,
              n_depths: int, depth_min_m: float, depth_max_m: float, *,
              wavelength_m: float = 0.0, cycles: float = 5.0, sigma_s: int = 2, sigma_t: int = 0,
              delta_m: float = 0.0, pad_factor: int = 2, c: float = C_LIGHT) -> PhasorPlan:
    """Plan-time quantities of the radial RSD operator (Sec. 4.3, supplementary)."""
    dx = wall_w_m / nx
    dy = wall_h_m / ny
    lam = wavelength_m if wavelength_m > 0 else 4.0 * dx
    band = virtual_wave_band(temporal_length(nt), bin_width_s, lam, cycles, c)
    lambda_min = c / band.freqs.max()
    Nu, Nv = _padded(nx, pad_factor), _padded(ny, pad_factor)
    rs = radial_sampling(Nu, Nv, dx, dy, sigma_s, lambda_min)
    depths = depth_planes(n_depths, depth_min_m, depth_max_m)
    kappa = 2.0 * np.pi * band.freqs / c                                   # [F]
    # A(r_j, d, f) = exp(i sigma_s kappa_f sqrt(r_j^2 + d^2))              (Eq. 4)
    R = np.sqrt(rs.r[:, None] ** 2 + depths[None, :] ** 2)                 # [N_r, D]
    A = np.exp(1j * sigma_s * kappa[None, :, None] * R[:, None, :])        # [N_r, F, D]
    K = ring_integral(A, rs.r, rs.q, rs.rho)                               # [N_rho, F, D]
    mod = np.exp(1j * kappa[:, None] * (sigma_t * depths[None, :] + delta_m))  # [F, D]
    K = K * mod[None, :, :]
    K[rs.rho > rs.rho_cut] = 0.0
    return PhasorPlan(nx, ny, nt, bin_width_s, wall_w_m, wall_h_m, pad_factor, dx, dy, Nu, Nv,
                      lam, cycles, band, lambda_min, sigma_s, sigma_t, delta_m, depths, rs, K)


def pixel_radius_bins(plan: PhasorPlan) -> np.ndarray:
    """Continuous radial bin coordinate rho~ of each DFT pixel (kx, ky)."""
    kx = np.arange(plan.Nu)
    ky = np.arange(plan.Nv)
    sx = np.where(kx < plan.Nu // 2, kx, kx - plan.Nu) / (plan.Nu * plan.dx)
    sy = np.where(ky < plan.Nv // 2, ky, ky - plan.Nv) / (plan.Nv * plan.dy)
    rho = np.sqrt(sx[:, None] ** 2 + sy[None, :] ** 2)
    return rho * (plan.radial.n_rho - 1) / plan.radial.rho_max


def phasor_field(H: np.ndarray, plan: PhasorPlan) -> np.ndarray:
    """P(x, y, f) = sum_t H(x, y, t) e^{-2 pi i k_f t / Lt} at the band bins
    (Lt = temporal_length(nt))."""
    H = np.asarray(H, dtype=np.float64)
    spec = sfft.rfft(H, n=temporal_length(H.shape[2]), axis=2, workers=_workers(None))
    return spec[:, :, plan.band.bins]


def propagate(P: np.ndarray, plan: PhasorPlan, workers=None) -> np.ndarray:
    """Alg. 4 applied to phasors P[x][y][f]: returns the complex I[x][y][d] (top-left a x b)."""
    a, b, F = P.shape
    Pp = np.zeros((plan.Nu, plan.Nv, F), dtype=np.complex128)
    Pp[:a, :b, :] = P
    Ph = sfft.fft2(Pp, axes=(0, 1), workers=_workers(workers))            # pad_tl + 2D DFTs
    rb = pixel_radius_bins(plan)
    acut = taper(rb, plan.radial.rho_cut_bin)
    i0, i1, alpha = lerp_indices(rb, plan.radial.rho_cut_bin, plan.radial.n_rho)
    w = plan.band.weights
    K = plan.K_r
    D = K.shape[2]
    C = np.zeros((plan.Nu * plan.Nv, D), dtype=np.complex128)
    Phf = Ph.reshape(-1, F)
    i0f, i1f, af, cf = i0.reshape(-1), i1.reshape(-1), alpha.reshape(-1), acut.reshape(-1)
    chunk = 512
    for s in range(0, Phf.shape[0], chunk):
        e = min(Phf.shape[0], s + chunk)
        al = af[s:e, None, None]
        h = cf[s:e, None, None] * ((1.0 - al) * K[i0f[s:e]] + al * K[i1f[s:e]])   # [p, F, D]
        C[s:e] = np.matmul((w[None, :] * Phf[s:e])[:, None, :], h)[:, 0, :]
    C = C.reshape(plan.Nu, plan.Nv, D)
    I = sfft.ifft2(C, axes=(0, 1), workers=_workers(workers))
    return I[:a, :b, :]


def pf_reconstruct(H: np.ndarray, plan: PhasorPlan, workers=None) -> np.ndarray:
    """|I| volume [x][y][d] of the radial phasor-field reconstruction."""
    return np.abs(propagate(phasor_field(H, plan), plan, workers))
