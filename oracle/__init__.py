"""FP64 CPU oracle for wave-based NLOS reconstruction.

TEST INFRASTRUCTURE ONLY. Only the tests, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` may import this package. The CUDA library never
calls it, and it shares no code, tables or constants with the CUDA path.

It is a plain, slow, obviously correct restatement of what the paper's hot path
computes, written from the paper in float64 with numpy/scipy:

  fk.py             confocal f-k migration (Sec. 3.1, Eq. 2; Alg. 1)
  pf.py             symmetry-aware phasor-field RSD reconstruction
                    (Sec. 4.3, Eqs. 3-7; supplementary radial sampling and
                    taper equations; Alg. 4)
  backprojection.py brute-force confocal backprojection (a comparison
                    baseline of Sec. 2), used only to pin peak locations
  rsd_direct.py     direct spatial Rayleigh-Sommerfeld summation (Eq. 3),
                    used only to pin peak locations of the radial operator
  post.py           max-over-depth images, mixture of experts (Eq. 10),
                    coherence merge (Eqs. 8-9), depth-dependent average
                    (Sec. 4.4)
  binning.py        photon binning into transients and compact phasors
                    (Sec. 4.1)

Library primitives used as single steps: scipy.fft (DFTs), scipy.special.j0
(Bessel J0), numpy matmul. Every function cites the passage it follows.
Parity status of each function is stated in its module header.
"""
