"""Pins of the photon-binning oracle (Sec. 4.1) against facts that do not
depend on it: count conservation, the window edges, round trips through
photon lists, and the FFT route to the phasor field."""
import numpy as np

from oracle import binning, pf
from paper_2608_28183_gb300 import synth


def test_histogram_round_trip_and_conservation():
    rng = np.random.default_rng(1)
    counts = rng.poisson(0.8, size=(6, 5, 32))
    s = synth.photons_from_counts(counts, ticks_per_bin=7, t0=50, seed=3, order="shuffled", stray=40)
    H = binning.bin_transient(s.pixel, s.ticks, 6, 5, 32, s.t0, s.ticks_per_bin)
    assert np.array_equal(H, counts)
    assert H.sum() == counts.sum() == len(s.pixel) - 40


def test_window_edges():
    nx, ny, nt, t0, tpb = 2, 3, 4, 100, 10
    pixel = np.array([0, 0, 0, 0, 5, 6, 1, 1], dtype=np.uint32)
    ticks = np.array([99, 100, 139, 140, 109, 100, 110, 119], dtype=np.uint32)
    H = binning.bin_transient(pixel, ticks, nx, ny, nt, t0, tpb)
    ref = np.zeros((nx, ny, nt))
    ref[0, 0, 0] += 1      # tick 100: first tick of bin 0
    ref[0, 0, 3] += 1      # tick 139: last tick of the last bin
    ref[1, 2, 0] += 1      # wall index 5 = (1, 2)
    ref[0, 1, 1] += 2      # ticks 110 and 119 share bin 1
    assert np.array_equal(H, ref)   # tick 99 (before t0), 140 (past the end), index 6 dropped


def test_phasors_equal_fft_of_histogram():
    """Direct per-photon accumulation vs w(f) * rFFT of the binned histogram."""
    g = synth.Geometry(8, 8, 128, 32e-12, 0.4, 0.4)
    plan = pf.make_plan(g.nx, g.ny, g.nt, g.bin_width_s, g.wall_w_m, g.wall_h_m, 4, 0.3, 0.6)
    rng = np.random.default_rng(5)
    counts = rng.poisson(1.5, size=(g.nx, g.ny, g.nt))
    s = synth.photons_from_counts(counts, seed=2, stray=25)
    P = binning.bin_phasors(s.pixel, s.ticks, g.nx, g.ny, g.nt, s.t0, s.ticks_per_bin, plan.band.bins, plan.band.weights)
    H = binning.bin_transient(s.pixel, s.ticks, g.nx, g.ny, g.nt, s.t0, s.ticks_per_bin)
    ref = pf.phasor_field(H, plan) * plan.band.weights[None, None, :]
    assert P.shape == (g.nx, g.ny, len(plan.band.bins))
    np.testing.assert_allclose(P, ref, rtol=0, atol=1e-9 * np.abs(ref).max())


def test_phasors_equal_fft_of_histogram_any_length():
    """Same identity on a temporal axis that is not a power of two (the
    phasor DFT runs over the zero-padded length)."""
    g = synth.Geometry(6, 5, 200, 32e-12, 0.3, 0.3)
    plan = pf.make_plan(g.nx, g.ny, g.nt, g.bin_width_s, g.wall_w_m, g.wall_h_m, 4, 0.3, 0.6)
    counts = np.random.default_rng(7).poisson(1.0, size=(g.nx, g.ny, g.nt))
    s = synth.photons_from_counts(counts, seed=4)
    P = binning.bin_phasors(s.pixel, s.ticks, g.nx, g.ny, g.nt, s.t0, s.ticks_per_bin, plan.band.bins,
                            plan.band.weights)
    ref = pf.phasor_field(binning.bin_transient(s.pixel, s.ticks, g.nx, g.ny, g.nt, s.t0, s.ticks_per_bin), plan)
    ref = ref * plan.band.weights[None, None, :]
    np.testing.assert_allclose(P, ref, rtol=0, atol=1e-9 * np.abs(ref).max())


def test_single_photon_phasor():
    """One photon in bin b gives w(f) exp(-2 pi i k_f b / n), the textbook DFT of a delta."""
    k = np.array([1, 5, 31])
    w = np.array([0.5, 1.0, 0.25])
    P = binning.bin_phasors(np.array([3], np.uint32), np.array([0 + 9 * 4], np.uint32), 2, 2, 64, 0, 4, k, w)
    b = 9
    assert np.allclose(P[1, 1], w * np.exp(-2j * np.pi * k * b / 64))
    assert np.count_nonzero(P) == 3
