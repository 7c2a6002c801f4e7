"""Cross-method pin: f-k and phasor-field oracles locate reflectors at the same
place in metres (within max(lateral voxel, depth-plane spacing))."""
import numpy as np
import pytest

from oracle import fk, pf
from paper_2608_28183_gb300 import synth

C = synth.C_LIGHT


@pytest.mark.parametrize("geom,pts", [
    (synth.Geometry(32, 32, 512, 16e-12, 1.0, 1.0), [(0.15, -0.1, 0.7), (-0.22, 0.18, 1.0)]),
    # padded to powers of two; the time window reaches 0.96 m
    (synth.Geometry(24, 28, 400, 16e-12, 0.9, 1.0), [(0.15, -0.1, 0.7), (-0.22, 0.18, 0.88)]),
])
def test_fk_and_pf_agree_on_reflector_position(geom, pts):
    xs = synth.wall_coords(geom.nx, geom.wall_w_m)
    ys = synth.wall_coords(geom.ny, geom.wall_h_m)
    p = pf.make_plan(geom.nx, geom.ny, geom.nt, geom.bin_width_s, geom.wall_w_m, geom.wall_h_m, 40, 0.4, 1.2)
    tol_x = geom.wall_w_m / geom.nx + 1e-9
    tol_y = geom.wall_h_m / geom.ny + 1e-9
    tol_z = max(p.depths[1] - p.depths[0], C * geom.bin_width_s / 2) + 1e-9
    for pt in pts:
        cap = synth.point_capture(geom, [(*pt, 1.0)])
        R = fk.fk_reconstruct(cap.counts, geom.bin_width_s, geom.wall_w_m, geom.wall_h_m)
        I = pf.pf_reconstruct(cap.counts, p)
        i, j, k = np.unravel_index(int(np.argmax(R)), R.shape)
        u, v, d = np.unravel_index(int(np.argmax(I)), I.shape)
        fk_pos = np.array([xs[i], ys[j], k * C * geom.bin_width_s / 2])
        pf_pos = np.array([xs[u], ys[v], p.depths[d]])
        assert abs(fk_pos[0] - pf_pos[0]) <= tol_x
        assert abs(fk_pos[1] - pf_pos[1]) <= tol_y
        assert abs(fk_pos[2] - pf_pos[2]) <= tol_z
