"""Post-processing of reconstructions in float64 (test infrastructure only).

Follows Sec. 4.4 (background-noise removal) and the display reduction of
Sec. 4.2 / Alg. 1:

  * max_image: the reduction to an image, f(x, y) = max_z v(x, y, z) of a
    magnitude volume (|Psi| for f-k, |I| for phasor fields).
  * moe_mix (Eq. 10): f = f_fk * (f_rsd + eps)^beta on the two branches'
    images. Reading: both images are first divided by their own maximum (the
    paper normalises displayed images; eps is then relative to the peak), and
    the mixture is divided by its maximum afterwards ("the mixed result is
    normalized").
  * coherence (Eq. 8) and coherent_merge (Eq. 9) over a window of N_w complex
    frames: C = |sum f_j| / (eps + sum |f_j|), merged = C |sum f_j| / N_w.
  * dda: depth-dependent average over the last N_w magnitude volumes. The
    paper states only that the weights depend on depth. Reading: a plane at
    depth index z averages the newest N(z) frames with
    N(z) = min(N_w, 1 + floor(N_w z / n_z)), so near planes (strong, early
    light) keep their temporal detail and far planes (weak, late light) are
    averaged over the full window.

Parity: pinned (tests/test_oracle_post.py): coherence bounds 0 <= C < 1,
C = 0 for frames that cancel and C -> 1 for identical frames, the merge of
identical frames equals |f| C; beta = 1 gives the plain product of the
normalised images and beta = 0 the f-k image; DDA with N_w = 1 is the
identity, a constant sequence is a fixed point, and a 3-frame x 4-depth case
matches values worked out by hand from the reading above (N = 1, 1, 2, 3).
"""
from __future__ import annotations

import numpy as np


def max_image(volume: np.ndarray) -> np.ndarray:
    """f(x, y) = max over the last (depth) axis."""
    return np.asarray(volume, dtype=np.float64).max(axis=-1)


def moe_mix(img_fk: np.ndarray, img_rsd: np.ndarray, beta: float = 0.3, eps: float = 1e-3) -> np.ndarray:
    """Eq. 10 on max-normalised images; the result is normalised to peak 1."""
    a = np.asarray(img_fk, dtype=np.float64)
    b = np.asarray(img_rsd, dtype=np.float64)
    a = a / a.max() if a.max() > 0 else a
    b = b / b.max() if b.max() > 0 else b
    f = a * (b + eps) ** beta
    return f / f.max() if f.max() > 0 else f


def coherence(frames: np.ndarray, eps: float = 1e-6) -> np.ndarray:
    """Eq. 8 over the first axis (the N_w frames)."""
    f = np.asarray(frames, dtype=np.complex128)
    return np.abs(f.sum(axis=0)) / (eps + np.abs(f).sum(axis=0))


def coherent_merge(frames: np.ndarray, eps: float = 1e-6) -> np.ndarray:
    """Eq. 9: C |sum f_j| / N_w."""
    f = np.asarray(frames, dtype=np.complex128)
    return coherence(f, eps) * np.abs(f.sum(axis=0)) / f.shape[0]


def dda_counts(nz: int, nw: int) -> np.ndarray:
    z = np.arange(nz)
    return np.minimum(nw, 1 + (nw * z) // nz)


def dda(frames: np.ndarray) -> np.ndarray:
    """Depth-dependent average; frames[0] is the newest of N_w volumes [.., nz]."""
    f = np.asarray(frames, dtype=np.float64)
    nw, nz = f.shape[0], f.shape[-1]
    counts = dda_counts(nz, nw)
    out = np.zeros(f.shape[1:])
    for z in range(nz):
        out[..., z] = f[: counts[z], ..., z].mean(axis=0)
    return out
