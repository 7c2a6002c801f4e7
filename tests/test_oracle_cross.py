"""Cross-method pin: f-k and phasor-field oracles locate reflectors at the same
place in metres (within max(lateral voxel, depth-plane spacing))."""
import numpy as np

from oracle import fk, pf
from paper_2608_28183_gb300 import synth

C = synth.C_LIGHT


def test_fk_and_pf_agree_on_reflector_position():
    geom = synth.Geometry(32, 32, 512, 16e-12, 1.0, 1.0)
    xs = synth.wall_coords(32, 1.0)
    p = pf.make_plan(32, 32, 512, 16e-12, 1.0, 1.0, 40, 0.4, 1.2)
    tol_lat = 1.0 / 32 + 1e-9
    tol_z = max(p.depths[1] - p.depths[0], C * 16e-12 / 2) + 1e-9
    for pt in [(0.15, -0.1, 0.7), (-0.22, 0.18, 1.0)]:
        cap = synth.point_capture(geom, [(*pt, 1.0)])
        R = fk.fk_reconstruct(cap.counts, geom.bin_width_s, 1.0, 1.0)
        I = pf.pf_reconstruct(cap.counts, p)
        i, j, k = np.unravel_index(int(np.argmax(R)), R.shape)
        u, v, d = np.unravel_index(int(np.argmax(I)), I.shape)
        fk_pos = np.array([xs[i], xs[j], k * C * 16e-12 / 2])
        pf_pos = np.array([xs[u], xs[v], p.depths[d]])
        assert abs(fk_pos[0] - pf_pos[0]) <= tol_lat
        assert abs(fk_pos[1] - pf_pos[1]) <= tol_lat
        assert abs(fk_pos[2] - pf_pos[2]) <= tol_z
