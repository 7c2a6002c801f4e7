"""GPU parity of the dense phasor-field method (Alg. 3) against the direct
Rayleigh-Sommerfeld sum of Eq. 3 in float64 (oracle/rsd_direct.py): with the
kernel sampled on the signed padded grid, the FFT convolution equals the
direct sum over wall samples, so the complex field must match to relative
L2 <= 1e-5."""
import numpy as np
import pytest

from oracle import pf, rsd_direct
from paper_2608_28183_gb300 import synth
from tests.gpu_util import exact_input, rel_l2, same_peak, to_device

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def library():
    from paper_2608_28183_gb300 import build, nlos
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return nlos.load_library()


def _capture(geom, seed, zr):
    rng = np.random.default_rng(seed)
    pts = [(rng.uniform(-0.3, 0.3) * geom.wall_w_m, rng.uniform(-0.3, 0.3) * geom.wall_h_m,
            rng.uniform(*zr), 1.0) for _ in range(2)]
    return synth.render(geom, synth.Scene(points=np.array(pts)), peak=300.0, background=0.5, seed=seed)


CASES = [
    (synth.Geometry(8, 8, 256, 32e-12, 0.4, 0.4), (5, 0.3, 0.9), (0.4, 0.9), {}),
    (synth.Geometry(16, 16, 256, 24e-12, 0.6, 0.6), (12, 0.3, 0.9), (0.4, 0.8), {}),
    (synth.Geometry(16, 8, 512, 16e-12, 0.8, 0.4), (9, 0.4, 1.0), (0.5, 0.9), {}),
    (synth.Geometry(16, 16, 256, 24e-12, 0.6, 0.6), (10, 0.3, 0.9), (0.4, 0.8),
     dict(sigma_s=1, sigma_t=1, delta_m=0.05)),
    (synth.Geometry(12, 10, 200, 32e-12, 0.5, 0.4), (7, 0.3, 0.9), (0.4, 0.8), {}),   # no power of two
]


@pytest.mark.parametrize("geom,depths,zr,kw", CASES, ids=["8x8", "16x16", "16x8", "16x16-nonconfocal", "12x10x200"])
def test_dense_matches_direct_rsd(geom, depths, zr, kw):
    from paper_2608_28183_gb300 import nlos
    D, dmin, dmax = depths
    plan = nlos.plan_for_capture(geom, "pf_dense", n_depths=D, depth_min_m=dmin, depth_max_m=dmax,
                                 output="complex", **kw)
    oplan = pf.make_plan(geom.nx, geom.ny, geom.nt, geom.bin_width_s, geom.wall_w_m, geom.wall_h_m, D, dmin, dmax,
                         **{k: v for k, v in kw.items() if v})
    cap = _capture(geom, geom.nx + geom.nt, zr)
    got = plan.reconstruct(to_device(cap.counts, torch.float32)).cpu().numpy().astype(np.complex128)
    P = pf.phasor_field(exact_input(cap.counts, torch.float32), oplan)
    ref = rsd_direct.rsd_direct(P, oplan.band.freqs, oplan.band.weights, oplan.depths, geom.wall_w_m, geom.wall_h_m,
                                sigma_s=kw.get("sigma_s", 2), sigma_t=kw.get("sigma_t", 0),
                                delta_m=kw.get("delta_m", 0.0))
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    assert same_peak(np.abs(got), np.abs(ref))


def test_dense_and_radial_find_the_same_reflectors():
    """The radial operator approximates the dense one (Sec. 4.3): same peak
    voxel to within one voxel on each axis."""
    from paper_2608_28183_gb300 import nlos
    geom = synth.Geometry(32, 32, 512, 16e-12, 1.0, 1.0)
    kw = dict(n_depths=40, depth_min_m=0.4, depth_max_m=1.2)
    cap = synth.point_capture(geom, [(0.12, -0.1, 0.75, 1.0)])
    x = to_device(cap.counts, torch.float32)
    dense = nlos.plan_for_capture(geom, "pf_dense", **kw).reconstruct(x).cpu().numpy()
    radial = nlos.plan_for_capture(geom, "pf", **kw).reconstruct(x).cpu().numpy()
    pd = np.unravel_index(np.argmax(dense), dense.shape)
    pr = np.unravel_index(np.argmax(radial), radial.shape)
    assert all(abs(int(u) - int(v)) <= 1 for u, v in zip(pd, pr)), (pd, pr)


def test_dense_workload_grid_sampled():
    """64 x 64 x 512 with 32 planes: magnitudes at sampled voxels against the
    oracle's direct sum evaluated at those voxels only."""
    from paper_2608_28183_gb300 import nlos
    geom = synth.Geometry(64, 64, 512, 16e-12, 1.0, 1.0)
    D, dmin, dmax = 32, 0.4, 1.2
    plan = nlos.plan_for_capture(geom, "pf_dense", n_depths=D, depth_min_m=dmin, depth_max_m=dmax)
    oplan = pf.make_plan(64, 64, 512, 16e-12, 1.0, 1.0, D, dmin, dmax)
    cap = _capture(geom, 9, (0.5, 1.0))
    vol = plan.reconstruct(to_device(cap.counts, torch.float32)).cpu().numpy().astype(np.float64)
    P = pf.phasor_field(exact_input(cap.counts, torch.float32), oplan)
    rng = np.random.default_rng(3)
    peak = np.unravel_index(np.argmax(vol), vol.shape)
    idx = [tuple(int(v) for v in peak)] + [(int(rng.integers(64)), int(rng.integers(64)), int(rng.integers(D)))
                                           for _ in range(24)]
    ref = np.abs(rsd_direct.rsd_direct_at(P, oplan.band.freqs, oplan.band.weights,
                                          [(i, j, oplan.depths[k]) for i, j, k in idx], 1.0, 1.0))
    got = np.array([vol[i] for i in idx])
    assert rel_l2(got, ref) <= 1e-5


def test_dense_rejects_half_storage():
    from paper_2608_28183_gb300 import nlos
    geom = synth.Geometry(16, 16, 256, 24e-12, 0.6, 0.6)
    with pytest.raises(nlos.NlosError, match="UNSUPPORTED"):
        nlos.plan_for_capture(geom, "pf_dense", "f16", n_depths=4, depth_min_m=0.3, depth_max_m=0.6)
