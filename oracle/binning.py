"""Photon binning in float64 (test infrastructure only).

Follows Sec. 4.1 (photon binner): a SPAD stream is a list of photon records,
each naming the relay-wall point it was detected at and its time of flight.
The binner either builds the transient histogram H(x, y, t) consumed by f-k
migration, or accumulates the photons directly into the compact phasor
field of the phasor-field pipeline (one complex value per wall point and
band frequency), which is the temporal Fourier transform of H at the band
bins, weighted by the virtual wave.

Record format (the library's, stated in its header): two uint32 arrays, the
wall index x * ny + y and the timestamp in integer ticks. Readings where the
paper is silent:

  * bin = (ticks - t0) // ticks_per_bin, in integers, so the decision is exact
    on both sides; photons with ticks < t0, bin >= nt or a wall index outside
    the grid are dropped.
  * The phasor of a photon in bin b at band bin k_f is exp(-2 pi i k_f b / Lt)
    with Lt the temporal DFT length of the phasor pipeline (nt, or the next
    power of two for other nt; the forward DFT sign of the phasor field); the
    compact phasor field is
    P[x][y][f] = w(f) * sum over the photons of (x, y) of that phasor, with
    w(f) the virtual-wave weight of the band (the same P the phasor pipeline
    forms from H).

Parity: pinned (tests/test_oracle_binning.py): photon counts are conserved,
records are dropped exactly at the window edges, histograms of photons made
from a histogram give it back, and the directly accumulated phasors equal
w(f) times the FFT of the binned histogram at the band bins (pf.phasor_field,
an independent route through scipy.fft).
"""
from __future__ import annotations

import numpy as np

from .pf import temporal_length


def bin_indices(pixel: np.ndarray, ticks: np.ndarray, nx: int, ny: int, nt: int, t0: int, ticks_per_bin: int):
    """(wall index, bin) of every photon kept by the time and grid window."""
    p = np.asarray(pixel, dtype=np.int64)
    t = np.asarray(ticks, dtype=np.int64) - int(t0)
    b = np.where(t >= 0, t // int(ticks_per_bin), -1)
    keep = (t >= 0) & (b < nt) & (p >= 0) & (p < nx * ny)
    return p[keep], b[keep]


def bin_transient(pixel, ticks, nx: int, ny: int, nt: int, t0: int, ticks_per_bin: int) -> np.ndarray:
    """H[x][y][t]: photon counts per wall point and time bin."""
    p, b = bin_indices(pixel, ticks, nx, ny, nt, t0, ticks_per_bin)
    H = np.zeros(nx * ny * nt, dtype=np.float64)
    np.add.at(H, p * nt + b, 1.0)
    return H.reshape(nx, ny, nt)


def bin_phasors(pixel, ticks, nx: int, ny: int, nt: int, t0: int, ticks_per_bin: int,
                band_bins: np.ndarray, band_w: np.ndarray) -> np.ndarray:
    """P[x][y][f] = w(f) * sum_photons exp(-2 pi i k_f b / Lt), accumulated per photon."""
    p, b = bin_indices(pixel, ticks, nx, ny, nt, t0, ticks_per_bin)
    Lt = temporal_length(nt)
    k = np.asarray(band_bins, dtype=np.int64)
    P = np.zeros((nx * ny, len(k)), dtype=np.complex128)
    step = 1 << 14
    for s in range(0, len(p), step):                     # one row of phasors per photon
        ph = np.exp(-2j * np.pi * np.outer(b[s:s + step], k) / Lt)
        np.add.at(P, p[s:s + step], ph)
    return (P * np.asarray(band_w, dtype=np.float64)[None, :]).reshape(nx, ny, len(k))
