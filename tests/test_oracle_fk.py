"""Pins of the FP64 f-k oracle against what the method and the mathematics fix.

None of these re-derive the oracle's own formulas: each compares it with a
closed form, a physical invariant (focusing of rendered point reflectors), an
independent brute-force method, or an independent discretisation of the same
Fourier integral.
"""
import math

import numpy as np
import pytest

from oracle import backprojection, fk
from paper_2608_28183_gb300 import synth

C = synth.C_LIGHT


def _peak(vol):
    return np.unravel_index(int(np.argmax(vol)), vol.shape)


def _expected_voxel(geom, x0, y0, z0):
    xs = synth.wall_coords(geom.nx, geom.wall_w_m)
    ys = synth.wall_coords(geom.ny, geom.wall_h_m)
    return (int(np.argmin(abs(xs - x0))), int(np.argmin(abs(ys - y0))),
            int(math.floor(2 * z0 / (C * geom.bin_width_s))))


def test_spectrum_parseval():
    """The forward DFT3 of the scaled, padded volume conserves energy (Parseval)."""
    rng = np.random.default_rng(0)
    H = rng.poisson(3.0, size=(6, 5, 16)).astype(float)
    U = fk.fk_spectrum(H)
    ramp = np.arange(16) / 15.0
    u2 = np.sum((H * ramp) ** 2)
    assert np.isclose(np.sum(abs(U) ** 2), U.size * u2, rtol=1e-12)


@pytest.mark.parametrize("t0", [3, 10, 17])
def test_impulse_closed_form_zero_lateral_factor(t0):
    """With s_x = s_y = 0 the Stolt map is the identity on Z > 0, and the
    reconstruction of a wall impulse is the positive-half (analytic) filter of
    the scaled impulse along t; its closed form is a geometric series:

        psi(z) = (t0/(n-1)) / Lt * sum_{m=1}^{Lt/2-1} exp(2 pi i m (z - t0) / Lt)

    at the impulse's wall sample, and 0 at every other wall sample, with Lt
    the padded temporal length (2n for power-of-two n, here the next power
    of two >= 2n = 48, i.e. 64).
    """
    a, b, n = 4, 3, 24
    x0, y0 = 2, 1
    H = np.zeros((a, b, n))
    H[x0, y0, t0] = 1.0
    psi = fk.fk_reconstruct(H, 0, 0, 0, lateral=(0.0, 0.0), return_complex=True)
    Lt = fk.padded_length(n, 2)
    assert Lt == 64
    M = Lt // 2 - 1
    z = np.arange(n)
    theta = 2 * np.pi * (z - t0) / Lt
    with np.errstate(invalid="ignore", divide="ignore"):
        geo = np.exp(1j * theta) * (1 - np.exp(1j * M * theta)) / (1 - np.exp(1j * theta))
    geo = np.where(z == t0, M, geo)
    expect = (t0 / (n - 1)) / Lt * geo
    np.testing.assert_allclose(psi[x0, y0], expect, atol=1e-14)
    others = np.ones((a, b), bool)
    others[x0, y0] = False
    assert np.max(abs(psi[others])) < 1e-14
    R = fk.fk_reconstruct(H, 0, 0, 0, lateral=(0.0, 0.0))
    assert np.isclose(R[x0, y0, t0], ((t0 / (n - 1)) * M / Lt) ** 2, rtol=1e-12)


@pytest.mark.parametrize("geom,pt", [
    (synth.Geometry(32, 32, 256, 32e-12, 1.0, 1.0), (0.1, -0.2, 0.7)),
    (synth.Geometry(32, 32, 256, 32e-12, 1.0, 1.0), (-0.3, 0.25, 1.0)),
    (synth.Geometry(24, 40, 256, 32e-12, 0.8, 1.3), (-0.15, 0.3, 0.6)),
    (synth.Geometry(20, 28, 200, 32e-12, 0.7, 0.9), (0.1, -0.15, 0.6)),      # no power-of-two axis
])
def test_point_reflector_peak(geom, pt):
    """A single rendered point reflector reconstructs to a peak within one
    voxel of its true position, on square and non-square walls."""
    cap = synth.point_capture(geom, [(*pt, 1.0)])
    R = fk.fk_reconstruct(cap.counts, geom.bin_width_s, geom.wall_w_m, geom.wall_h_m)
    got = _peak(R)
    exp = _expected_voxel(geom, *pt)
    assert all(abs(g - e) <= 1 for g, e in zip(got, exp)), (got, exp)


def test_focus_is_sharpest_at_physical_lateral_factor():
    """The lateral factor s = c dt / (2 dx) is the one that focuses a rendered
    point target: scaling it up or down lowers the peak."""
    geom = synth.Geometry(32, 32, 256, 32e-12, 1.0, 1.0)
    cap = synth.point_capture(geom, [(0.1, -0.2, 0.7, 1.0)])
    sx, sy = fk.lateral_factors(geom.bin_width_s, geom.wall_w_m, geom.wall_h_m, 32, 32)
    assert np.isclose(sx, C * 32e-12 / (2 * (1.0 / 32)))
    peaks = {f: fk.fk_reconstruct(cap.counts, 0, 0, 0, lateral=(sx * f, sy * f)).max()
             for f in (0.8, 1.0, 1.25)}
    assert peaks[1.0] > 2.0 * max(peaks[0.8], peaks[1.25])


def test_lateral_factors_follow_their_own_axis():
    """On a wall whose pitches differ threefold (dx = 3 dy), the per-axis
    factors from the geometry focus a point; exchanging them does not."""
    geom = synth.Geometry(16, 48, 256, 32e-12, 1.0, 1.0)
    cap = synth.point_capture(geom, [(0.1, -0.15, 0.7, 1.0)])
    sx, sy = fk.lateral_factors(geom.bin_width_s, geom.wall_w_m, geom.wall_h_m, 16, 48)
    R = fk.fk_reconstruct(cap.counts, geom.bin_width_s, geom.wall_w_m, geom.wall_h_m)
    Rswap = fk.fk_reconstruct(cap.counts, 0, 0, 0, lateral=(sy, sx))
    assert R.max() > 2.0 * Rswap.max()
    exp = _expected_voxel(geom, 0.1, -0.15, 0.7)
    assert all(abs(g - e) <= 1 for g, e in zip(_peak(R), exp))


@pytest.mark.parametrize("geom", [synth.Geometry(8, 8, 64, 64e-12, 0.6, 0.6),
                                  synth.Geometry(10, 12, 96, 64e-12, 0.6, 0.7)])
def test_agrees_with_backprojection_peaks(geom):
    """On 8 x 8 x 64 and 10 x 12 x 96 grids (the latter padded to the next
    powers of two), f-k and brute-force backprojection put the peak of each
    rendered point reflector at the same voxel (within one voxel)."""
    for pt in [(0.05, -0.1, 0.6), (-0.15, 0.12, 0.9)]:
        cap = synth.point_capture(geom, [(*pt, 1.0)])
        R = fk.fk_reconstruct(cap.counts, geom.bin_width_s, geom.wall_w_m, geom.wall_h_m)
        B = backprojection.backproject(cap.counts, geom.bin_width_s, geom.wall_w_m, geom.wall_h_m)
        pf, pb = _peak(R), _peak(B)
        assert all(abs(i - j) <= 1 for i, j in zip(pf, pb)), (pf, pb)


def _continuous_stolt_reference(H, sx, sy, over=32):
    """Independent discretisation of the same Fourier integral.

    The oracle sums V(m~) = U(mu(m~)) (m~/mu) over integer m~ with U linearly
    interpolated. Changing the integration variable from m~ to the source
    coordinate k = mu gives int U(k) exp(2 pi i m~(k) z / Pt) dk with
    m~(k) = sqrt(k^2 - A): no weight, because the Jacobian factor cancels
    dm~/dk = k/m~. This evaluates that integral with the exact band-limited
    U(k) (direct DFT at fractional k) on a fine midpoint grid, starting at
    m~ = 1/2 (the lower edge of the oracle's first sample) and ending at the
    last sampled frequency Pt/2 - 1.
    """
    a, b, n = H.shape
    Px, Py, Pt = 2 * a, 2 * b, 2 * n
    u = np.zeros((Px, Py, n))
    u[:a, :b, :] = H * (np.arange(n) / (n - 1))
    Uxy = np.fft.fft2(u, axes=(0, 1))
    sgn = lambda N: np.where(np.arange(N) < N // 2, np.arange(N), np.arange(N) - N)
    X, Y = sgn(Px) / a, sgn(Py) / b
    dk = 1.0 / over
    zs, xs, ys = np.arange(n), np.arange(a), np.arange(b)
    psi = np.zeros((a, b, n), complex)
    for p in range(Px):
        for q in range(Py):
            A = (n * sx * X[p]) ** 2 + (n * sy * Y[q]) ** 2
            k_lo = np.sqrt(A + 0.25)
            if k_lo >= n - 1:
                continue
            k = np.arange(k_lo, n - 1, dk) + dk / 2
            Uk = np.exp(-2j * np.pi * np.outer(k, np.arange(n)) / Pt) @ Uxy[p, q]
            mt = np.sqrt(k * k - A)
            col = np.exp(2j * np.pi * np.outer(zs, mt) / Pt) @ (Uk * dk)
            ph = np.exp(2j * np.pi * (p * xs[:, None] / Px + q * ys[None, :] / Py))
            psi += ph[:, :, None] * col[None, None, :]
    return psi / (Px * Py * Pt)


@pytest.mark.parametrize("s", [0.3, 0.8])
def test_stolt_matches_continuous_integral(s):
    """Interpolated Stolt + Jacobian agrees with the interpolation-free
    evaluation of the same integral to ~1% on smooth early pulses (dropping or
    inverting the Jacobian gives 15-50% here)."""
    rng = np.random.default_rng(3)
    a = b = 4
    n = 64
    t = np.arange(n)
    H = np.zeros((a, b, n))
    for x in range(a):
        for y in range(b):
            t0 = rng.uniform(1.5, 3.5)
            H[x, y] = rng.uniform(0.2, 1) * np.exp(-(t - t0) ** 2 / (2 * 2.0 ** 2))
    psi = fk.fk_reconstruct(H, 0, 0, 0, lateral=(s, s), return_complex=True)
    ref = _continuous_stolt_reference(H, s, s)
    err = np.linalg.norm(psi - ref) / np.linalg.norm(ref)
    assert err < 0.03, err


def test_linear_before_magnitude():
    """Psi is linear in H (only |.|^2 at the end is not)."""
    rng = np.random.default_rng(1)
    H1 = rng.random((5, 6, 20))
    H2 = rng.random((5, 6, 20))
    args = (32e-12, 0.5, 0.6)
    p1 = fk.fk_reconstruct(H1, *args, return_complex=True)
    p2 = fk.fk_reconstruct(H2, *args, return_complex=True)
    p12 = fk.fk_reconstruct(2 * H1 - 3 * H2, *args, return_complex=True)
    np.testing.assert_allclose(p12, 2 * p1 - 3 * p2, atol=1e-12 * np.abs(p12).max())
