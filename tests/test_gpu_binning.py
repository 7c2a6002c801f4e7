"""GPU parity of photon binning (Sec. 4.1) through the C ABI: histograms are
bit-exact against the oracle; phasors and reconstructions from phasors match
the float64 oracle to relative L2 <= 1e-5."""
import numpy as np
import pytest

from oracle import binning, pf
from paper_2608_28183_gb300 import synth
from tests.gpu_util import rel_l2, same_peak

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def library():
    from paper_2608_28183_gb300 import build, nlos
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return nlos.load_library()


GEOM = synth.Geometry(32, 16, 256, 24e-12, 0.8, 0.4)
DEPTHS = (40, 0.4, 1.2)


def _dev(stream):
    return torch.from_numpy(stream.pixel).cuda(), torch.from_numpy(stream.ticks).cuda()


def _stream(geom, seed, order, stray=300, peak=40.0):
    rng = np.random.default_rng(seed)
    pts = [(rng.uniform(-0.3, 0.3) * geom.wall_w_m, rng.uniform(-0.3, 0.3) * geom.wall_h_m,
            rng.uniform(0.3, 0.8) * geom.nt * geom.bin_depth_m, 1.0) for _ in range(3)]
    cap = synth.render(geom, synth.Scene(points=np.array(pts)), peak=peak, background=0.5, seed=seed)
    return synth.photons_from_counts(cap.counts, ticks_per_bin=11, t0=500, seed=seed, order=order, stray=stray)


def _pf_plans(geom, **kw):
    from paper_2608_28183_gb300 import nlos
    D, dmin, dmax = DEPTHS
    plan = nlos.plan_for_capture(geom, "pf", n_depths=D, depth_min_m=dmin, depth_max_m=dmax, **kw)
    oplan = pf.make_plan(geom.nx, geom.ny, geom.nt, geom.bin_width_s, geom.wall_w_m, geom.wall_h_m, D, dmin, dmax)
    return plan, oplan


@pytest.mark.parametrize("order", ["scan", "shuffled"])
def test_bin_transient_exact(order):
    from paper_2608_28183_gb300 import nlos
    g = GEOM
    s = _stream(g, 3, order)
    px, tk = _dev(s)
    H = nlos.bin_transient(px, tk, g.nx, g.ny, g.nt, s.t0, s.ticks_per_bin).cpu().numpy()
    ref = binning.bin_transient(s.pixel, s.ticks, g.nx, g.ny, g.nt, s.t0, s.ticks_per_bin)
    assert np.array_equal(H, ref.astype(np.float32))


def test_bin_transient_accumulates_batches():
    from paper_2608_28183_gb300 import nlos
    g = GEOM
    s = _stream(g, 4, "shuffled")
    px, tk = _dev(s)
    h = px.numel() // 3
    H = nlos.bin_transient(px[:h], tk[:h], g.nx, g.ny, g.nt, s.t0, s.ticks_per_bin)
    nlos.bin_transient(px[h:], tk[h:], g.nx, g.ny, g.nt, s.t0, s.ticks_per_bin, transient=H, accumulate=True)
    ref = binning.bin_transient(s.pixel, s.ticks, g.nx, g.ny, g.nt, s.t0, s.ticks_per_bin)
    assert np.array_equal(H.cpu().numpy(), ref.astype(np.float32))


def test_bin_empty_and_all_stray():
    from paper_2608_28183_gb300 import nlos
    g = GEOM
    H = torch.ones((g.nx, g.ny, g.nt), device="cuda")
    e = torch.zeros(0, dtype=torch.uint32, device="cuda")
    nlos.bin_transient(e, e, g.nx, g.ny, g.nt, 0, 4, transient=H)
    assert float(H.abs().sum()) == 0.0
    px = torch.tensor([g.nx * g.ny, 3, 3], dtype=torch.uint32, device="cuda")
    tk = torch.tensor([0, 1, 4 * g.nt + 7], dtype=torch.uint32, device="cuda")   # off-grid, before t0, past the end
    nlos.bin_transient(px, tk, g.nx, g.ny, g.nt, 2, 4, transient=H)
    assert float(H.abs().sum()) == 0.0


@pytest.mark.parametrize("route", ["direct", "histogram", "auto"])
@pytest.mark.parametrize("order", ["scan", "shuffled"])
def test_bin_phasors_parity(order, route):
    g = GEOM
    plan, oplan = _pf_plans(g)
    k_lo, F = plan.band
    assert k_lo == oplan.band.bins[0] and F == len(oplan.band.bins)
    s = _stream(g, 5, order)
    px, tk = _dev(s)
    P = plan.bin_phasors(px, tk, s.t0, s.ticks_per_bin, route=route).cpu().numpy()
    ref = binning.bin_phasors(s.pixel, s.ticks, g.nx, g.ny, g.nt, s.t0, s.ticks_per_bin,
                              oplan.band.bins, oplan.band.weights)
    assert np.linalg.norm(P - ref) / np.linalg.norm(ref) <= 1e-5


@pytest.mark.parametrize("route", ["direct", "histogram"])
def test_bin_phasors_accumulate(route):
    g = GEOM
    plan, oplan = _pf_plans(g)
    s = _stream(g, 8, "shuffled")
    px, tk = _dev(s)
    h = px.numel() // 2
    P = plan.bin_phasors(px[:h], tk[:h], s.t0, s.ticks_per_bin, route=route)
    plan.bin_phasors(px[h:], tk[h:], s.t0, s.ticks_per_bin, phasors=P, accumulate=True, route=route)
    ref = binning.bin_phasors(s.pixel, s.ticks, g.nx, g.ny, g.nt, s.t0, s.ticks_per_bin,
                              oplan.band.bins, oplan.band.weights)
    got = P.cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5


@pytest.mark.parametrize("route", ["direct", "histogram"])
def test_bin_phasors_any_length(route):
    """A temporal axis that is not a power of two: the phasors are taken over
    the zero-padded DFT length."""
    from paper_2608_28183_gb300 import nlos
    g = synth.Geometry(20, 12, 200, 32e-12, 0.7, 0.4)
    plan = nlos.plan_for_capture(g, "pf", n_depths=8, depth_min_m=0.3, depth_max_m=0.9)
    oplan = pf.make_plan(g.nx, g.ny, g.nt, g.bin_width_s, g.wall_w_m, g.wall_h_m, 8, 0.3, 0.9)
    assert plan.band == (int(oplan.band.bins[0]), len(oplan.band.bins))
    s = _stream(g, 12, "shuffled")
    px, tk = _dev(s)
    P = plan.bin_phasors(px, tk, s.t0, s.ticks_per_bin, route=route).cpu().numpy()
    ref = binning.bin_phasors(s.pixel, s.ticks, g.nx, g.ny, g.nt, s.t0, s.ticks_per_bin,
                              oplan.band.bins, oplan.band.weights)
    assert np.linalg.norm(P - ref) / np.linalg.norm(ref) <= 1e-5


def test_reconstruct_from_binned_phasors():
    """Photons -> phasors -> volume equals photons -> histogram -> volume, and the oracle."""
    from paper_2608_28183_gb300 import nlos
    g = GEOM
    plan, oplan = _pf_plans(g)
    s = _stream(g, 6, "scan", peak=200.0)
    px, tk = _dev(s)
    vol_p = plan.reconstruct_phasors(plan.bin_phasors(px, tk, s.t0, s.ticks_per_bin))
    H = nlos.bin_transient(px, tk, g.nx, g.ny, g.nt, s.t0, s.ticks_per_bin)
    vol_h = plan.reconstruct(H)
    torch.cuda.synchronize()
    a, b = vol_p.cpu().numpy(), vol_h.cpu().numpy()
    ref = pf.pf_reconstruct(binning.bin_transient(s.pixel, s.ticks, g.nx, g.ny, g.nt, s.t0, s.ticks_per_bin), oplan)
    assert rel_l2(a, ref) <= 1e-5 and rel_l2(b, ref) <= 1e-5
    assert same_peak(a, ref)


def test_bin_phasors_full_workload_sampled():
    """128 x 128 x 1024 grid, a 1.2M-photon frame (the paper's frame size):
    all phasors against the histogram route, sampled wall points against the
    oracle's per-photon sum."""
    from paper_2608_28183_gb300 import nlos
    cap = synth.make_capture("pf_128x128x1024", 0, noise=False)
    g = cap.geometry
    plan = nlos.plan_for_capture(g, "pf", n_depths=128, depth_min_m=0.5, depth_max_m=2.5)
    oplan = pf.make_plan(g.nx, g.ny, g.nt, g.bin_width_s, g.wall_w_m, g.wall_h_m, 128, 0.5, 2.5)
    s = synth.photon_frame(cap, 1_200_000, seed=1)
    px, tk = _dev(s)
    P = plan.bin_phasors(px, tk, s.t0, s.ticks_per_bin).cpu().numpy()
    Pd = plan.bin_phasors(px, tk, s.t0, s.ticks_per_bin, route="direct").cpu().numpy()
    assert np.linalg.norm(P - Pd) / np.linalg.norm(Pd) <= 1e-5
    rng = np.random.default_rng(0)
    pick = rng.choice(g.nx * g.ny, size=64, replace=False)
    sel = np.isin(s.pixel, pick)
    ref = binning.bin_phasors(s.pixel[sel], s.ticks[sel], g.nx, g.ny, g.nt, s.t0, s.ticks_per_bin,
                              oplan.band.bins, oplan.band.weights).reshape(g.nx * g.ny, -1)[pick]
    got = P.reshape(g.nx * g.ny, -1)[pick]
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    H = nlos.bin_transient(px, tk, g.nx, g.ny, g.nt, s.t0, s.ticks_per_bin).cpu().numpy().astype(np.float64)
    assert H.sum() == len(s.pixel)
    hp = (pf.phasor_field(H, oplan) * oplan.band.weights[None, None, :])
    assert np.linalg.norm(P - hp) / np.linalg.norm(hp) <= 1e-5


def test_binning_rejects_bad_arguments():
    from paper_2608_28183_gb300 import nlos
    g = GEOM
    plan, _ = _pf_plans(g)
    px = torch.zeros(4, dtype=torch.uint32, device="cuda")
    with pytest.raises(nlos.NlosError, match="INVALID_ARG"):
        nlos.bin_transient(px, px, g.nx, g.ny, g.nt, 0, 0)
    with pytest.raises(nlos.NlosError, match="INVALID_ARG"):
        plan.bin_phasors(px, px, 0, 0)
    lib = nlos.load_library()
    with pytest.raises(nlos.NlosError, match="INVALID_ARG"):      # both routes forced at once
        nlos._check(lib.nlos_bin_phasors(plan.handle, px.data_ptr(), px.data_ptr(), 4, 0, 1, 6,
                                               plan.empty_phasors().data_ptr(), None))
    fkp = nlos.plan_for_capture(g, "fk")
    with pytest.raises(nlos.NlosError, match="INVALID_ARG"):
        _ = fkp.band
    half, _ = _pf_plans(g, storage="f16")
    with pytest.raises(nlos.NlosError, match="UNSUPPORTED"):
        half.reconstruct_phasors(plan.empty_phasors())
