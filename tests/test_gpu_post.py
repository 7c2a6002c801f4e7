"""GPU parity of the post-processing calls and of complex-output plans
against the FP64 oracle: max-over-depth images, the mixture of experts of
Eq. 10, the coherence merge of Eqs. 8-9 and the depth-dependent average."""
import numpy as np
import pytest

from oracle import fk, pf, post
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


GEOM = synth.Geometry(32, 32, 256, 24e-12, 0.8, 0.8)
DEPTHS = (48, 0.4, 1.2)


def _scene(geom, seed):
    rng = np.random.default_rng(seed)
    pts = [(rng.uniform(-0.3, 0.3) * geom.wall_w_m, rng.uniform(-0.3, 0.3) * geom.wall_h_m,
            rng.uniform(0.3, 0.8) * geom.nt * geom.bin_depth_m, 1.0) for _ in range(3)]
    return synth.Scene(points=np.array(pts))


def _frames(geom, nw, seed=3, peak=60.0):
    """N_w captures of one scene with independent photon noise."""
    scene = _scene(geom, seed)
    return [synth.render(geom, scene, peak=peak, background=0.5, seed=seed * 100 + j).counts for j in range(nw)]


def _run(plan, H):
    out = plan.reconstruct(to_device(H, plan.input_dtype()))
    torch.cuda.synchronize()
    return out


def test_fk_complex_output_parity():
    from paper_2608_28183_gb300 import nlos
    H = _frames(GEOM, 1)[0]
    plan = nlos.plan_for_capture(GEOM, "fk", output="complex")
    mag = nlos.plan_for_capture(GEOM, "fk")
    assert plan.output_bytes == 2 * mag.output_bytes
    got = _run(plan, H).cpu().numpy().astype(np.complex128)
    ref = fk.fk_reconstruct(exact_input(H, torch.float32), GEOM.bin_width_s, GEOM.wall_w_m, GEOM.wall_h_m,
                            return_complex=True)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    m = _run(mag, H).cpu().numpy().astype(np.float64)
    assert rel_l2(np.abs(got) ** 2, m) <= 1e-5


def test_fk_complex_output_half_storage():
    from paper_2608_28183_gb300 import nlos
    H = _frames(GEOM, 1, seed=5)[0]
    plan = nlos.plan_for_capture(GEOM, "fk", "f16", output="complex")
    got = _run(plan, H).cpu().numpy().astype(np.complex128)
    ref = fk.fk_reconstruct(exact_input(H, torch.float16), GEOM.bin_width_s, GEOM.wall_w_m, GEOM.wall_h_m,
                            return_complex=True)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 2e-3


def test_pf_complex_output_parity():
    from paper_2608_28183_gb300 import nlos
    D, dmin, dmax = DEPTHS
    H = _frames(GEOM, 1, seed=7)[0]
    plan = nlos.plan_for_capture(GEOM, "pf", n_depths=D, depth_min_m=dmin, depth_max_m=dmax, output="complex")
    oplan = pf.make_plan(GEOM.nx, GEOM.ny, GEOM.nt, GEOM.bin_width_s, GEOM.wall_w_m, GEOM.wall_h_m, D, dmin, dmax)
    got = _run(plan, H).cpu().numpy().astype(np.complex128)
    ref = pf.propagate(pf.phasor_field(exact_input(H, torch.float32), oplan), oplan)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5


@pytest.mark.parametrize("shape", [(32, 32, 256), (8, 16, 7), (3, 5, 100), (1, 1, 1), (64, 64, 33)])
@pytest.mark.parametrize("take_sqrt", [False, True])
def test_max_image(shape, take_sqrt):
    from paper_2608_28183_gb300 import nlos
    rng = np.random.default_rng(sum(shape))
    v = rng.gamma(0.5, size=shape).astype(np.float32)
    img = nlos.max_image(torch.from_numpy(v).cuda(), take_sqrt=take_sqrt).cpu().numpy()
    ref = post.max_image(v)
    if take_sqrt:
        ref = np.sqrt(ref)
        np.testing.assert_allclose(img, ref, rtol=1e-6)
    else:
        assert np.array_equal(img, ref.astype(np.float32))   # a max is exact


def test_moe_on_reconstructions():
    """The whole branch mix: f-k |Psi| image and phasor |I| image of one capture, Eq. 10."""
    from paper_2608_28183_gb300 import nlos
    D, dmin, dmax = DEPTHS
    H = _frames(GEOM, 1, seed=11, peak=300.0)[0]
    Hx = exact_input(H, torch.float32)
    fkp = nlos.plan_for_capture(GEOM, "fk")
    pfp = nlos.plan_for_capture(GEOM, "pf", n_depths=D, depth_min_m=dmin, depth_max_m=dmax)
    x = to_device(H, torch.float32)
    img_fk = nlos.max_image(fkp.reconstruct(x), take_sqrt=True)
    img_rsd = nlos.max_image(pfp.reconstruct(x))
    mix = nlos.moe_mix(img_fk, img_rsd, beta=0.3, eps=1e-3).cpu().numpy()
    oplan = pf.make_plan(GEOM.nx, GEOM.ny, GEOM.nt, GEOM.bin_width_s, GEOM.wall_w_m, GEOM.wall_h_m, D, dmin, dmax)
    ref_fk = np.sqrt(post.max_image(fk.fk_reconstruct(Hx, GEOM.bin_width_s, GEOM.wall_w_m, GEOM.wall_h_m)))
    ref_rsd = post.max_image(pf.pf_reconstruct(Hx, oplan))
    ref = post.moe_mix(ref_fk, ref_rsd, beta=0.3, eps=1e-3)
    assert rel_l2(mix, ref) <= 1e-5
    assert same_peak(mix, ref)
    assert abs(mix.max() - 1.0) <= 1e-6


@pytest.mark.parametrize("n,beta,eps", [(1, 0.3, 1e-3), (1000, 0.3, 1e-3), (128 * 128, 1.0, 0.0),
                                        (70001, 0.0, 1e-3), (256 * 256, 0.7, 0.05)])
def test_moe_sizes(n, beta, eps):
    from paper_2608_28183_gb300 import nlos
    rng = np.random.default_rng(n)
    a = rng.gamma(0.7, size=n).astype(np.float32)
    b = rng.gamma(0.7, size=n).astype(np.float32)
    got = nlos.moe_mix(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), beta=beta, eps=eps).cpu().numpy()
    ref = post.moe_mix(a, b, beta=beta, eps=eps)
    np.testing.assert_allclose(got, ref, rtol=2e-6, atol=2e-7)


@pytest.mark.parametrize("nw", [1, 4, 16])
def test_coherence_merge_of_reconstructions(nw):
    """Eqs. 8-9 over N_w noisy complex f-k reconstructions of one scene."""
    from paper_2608_28183_gb300 import nlos
    plan = nlos.plan_for_capture(GEOM, "fk", output="complex")
    caps = _frames(GEOM, nw, seed=13)
    vols = [plan.reconstruct(to_device(H, torch.float32)) for H in caps]
    merged, coh = nlos.coherence_merge(vols, eps=1e-6)
    torch.cuda.synchronize()
    frames = np.stack([v.cpu().numpy().astype(np.complex128) for v in vols])   # the same inputs for both sides
    ref_m = post.coherent_merge(frames, eps=1e-6)
    ref_c = post.coherence(frames, eps=1e-6)
    assert rel_l2(merged.cpu().numpy(), ref_m) <= 1e-5
    assert np.max(np.abs(coh.cpu().numpy() - ref_c)) <= 1e-5
    assert same_peak(merged.cpu().numpy(), ref_m)


def test_coherence_merge_ragged_and_bounds():
    from paper_2608_28183_gb300 import nlos
    rng = np.random.default_rng(2)
    n = 300007
    fr = [(rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64) for _ in range(5)]
    got_m, got_c = nlos.coherence_merge([torch.from_numpy(f).cuda() for f in fr], eps=1e-3)
    ref = np.stack(fr).astype(np.complex128)
    np.testing.assert_allclose(got_m.cpu().numpy(), post.coherent_merge(ref, 1e-3), rtol=1e-5, atol=1e-6)
    c = got_c.cpu().numpy()
    np.testing.assert_allclose(c, post.coherence(ref, 1e-3), rtol=1e-5, atol=1e-6)
    assert c.min() >= 0.0 and c.max() < 1.0


@pytest.mark.parametrize("nw,shape", [(1, (8, 8, 16)), (3, (16, 8, 37)), (8, (32, 32, 256)), (16, (5, 3, 64))])
def test_dda(nw, shape):
    from paper_2608_28183_gb300 import nlos
    rng = np.random.default_rng(nw)
    fr = [rng.gamma(0.5, size=shape).astype(np.float32) for _ in range(nw)]
    got = nlos.dda([torch.from_numpy(f).cuda() for f in fr]).cpu().numpy()
    ref = post.dda(np.stack(fr))
    np.testing.assert_allclose(got, ref, rtol=2e-6, atol=1e-7)
    if nw == 1:
        assert np.array_equal(got, fr[0])


def test_post_rejects_bad_arguments():
    from paper_2608_28183_gb300 import nlos
    v = torch.zeros(17 * 4, dtype=torch.complex64, device="cuda")
    with pytest.raises(nlos.NlosError, match="INVALID_ARG"):
        nlos.coherence_merge([v] * 17)
    with pytest.raises(nlos.NlosError, match="INVALID_ARG"):
        nlos.coherence_merge([v], eps=0.0)
    r = torch.zeros((4, 4, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(nlos.NlosError, match="INVALID_ARG"):
        nlos.dda([r] * 17)
    with pytest.raises(nlos.NlosError, match="INVALID_ARG"):
        nlos.moe_mix(r, r, eps=-1.0)


# the mixture's two experts from one shared lateral spectrum (Sec. 4.4):
# geometry, phasor method, f-k lateral stages separate, two streams, f-k output
SHARED = [
    (GEOM, "pf", False, True, "magnitude"),
    (GEOM, "pf", True, False, "magnitude"),
    (synth.Geometry(48, 64, 160, 24e-12, 0.8, 1.0), "pf", False, True, "complex"),
    (synth.Geometry(16, 16, 200, 24e-12, 0.6, 0.6), "pf_dense", False, True, "magnitude"),
]


@pytest.mark.parametrize("geom,method,sep,two,fk_out", SHARED,
                         ids=["32x32-fused-2streams", "32x32-separate-1stream", "48x64x160-complex",
                              "16x16x200-dense"])
def test_moe_shared_spectrum(geom, method, sep, two, fk_out):
    """Both experts from one x/y forward transform: each volume matches the
    oracle and the plan's own reconstruction of the same transient."""
    from oracle import rsd_direct
    from paper_2608_28183_gb300 import nlos
    D, dmin, dmax = DEPTHS
    H = _frames(geom, 1, seed=17, peak=300.0)[0]
    Hx = exact_input(H, torch.float32)
    fkp = nlos.plan_for_capture(geom, "fk", separate_axes=sep, output=fk_out)
    pfp = nlos.plan_for_capture(geom, method, n_depths=D, depth_min_m=dmin, depth_max_m=dmax)
    x = to_device(H, torch.float32)
    s2 = torch.cuda.Stream() if two else None
    for _ in range(2):                  # the second call reuses both workspaces and the events
        vf, vp = nlos.reconstruct_moe(fkp, pfp, x, stream2=s2)
    torch.cuda.synchronize()
    cpx = fk_out == "complex"
    got_fk = vf.cpu().numpy().astype(np.complex128 if cpx else np.float64)
    got_pf = vp.cpu().numpy().astype(np.float64)
    ref_fk = fk.fk_reconstruct(Hx, geom.bin_width_s, geom.wall_w_m, geom.wall_h_m, return_complex=cpx)
    assert np.linalg.norm(got_fk - ref_fk) / np.linalg.norm(ref_fk) <= 1e-5
    oplan = pf.make_plan(geom.nx, geom.ny, geom.nt, geom.bin_width_s, geom.wall_w_m, geom.wall_h_m, D, dmin, dmax)
    if method == "pf":
        ref_pf = pf.pf_reconstruct(Hx, oplan)
    else:
        P = pf.phasor_field(Hx, oplan)
        ref_pf = np.abs(rsd_direct.rsd_direct(P, oplan.band.freqs, oplan.band.weights, oplan.depths,
                                              geom.wall_w_m, geom.wall_h_m))
    assert rel_l2(got_pf, ref_pf) <= 1e-5
    assert same_peak(got_pf, ref_pf)
    # against each plan's own path on the same transient
    own_fk = fkp.reconstruct(x).cpu().numpy()
    own_pf = pfp.reconstruct(x).cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got_fk - own_fk) / np.linalg.norm(own_fk) <= 2e-6
    assert rel_l2(got_pf, own_pf) <= 2e-6


def test_moe_shared_spectrum_rejects_mismatched_plans():
    """The C entry refuses plans it cannot share a spectrum between (status
    codes, nothing launched); a zero transient gives zero volumes."""
    import ctypes
    from paper_2608_28183_gb300 import nlos
    D, dmin, dmax = DEPTHS
    fkp = nlos.plan_for_capture(GEOM, "fk")
    pfp = nlos.plan_for_capture(GEOM, "pf", n_depths=D, depth_min_m=dmin, depth_max_m=dmax)
    x = torch.zeros((GEOM.nx, GEOM.ny, GEOM.nt), device="cuda")
    vf, vp = fkp.empty_volume(), pfp.empty_volume()
    other = nlos.plan_for_capture(synth.Geometry(32, 32, 128, 24e-12, 0.8, 0.8), "pf", n_depths=D,
                                  depth_min_m=dmin, depth_max_m=dmax)
    half = nlos.plan_for_capture(GEOM, "pf", "f16", n_depths=D, depth_min_m=dmin, depth_max_m=dmax)

    def call(a, b):
        return nlos._lib.nlos_reconstruct_moe(a._h, b._h, ctypes.c_void_p(x.data_ptr()),
                                              ctypes.c_void_p(vf.data_ptr()), ctypes.c_void_p(vp.data_ptr()),
                                              None, None)
    invalid, unsupported = 1, 4
    assert nlos.STATUS[invalid] == "INVALID_ARG" and nlos.STATUS[unsupported] == "UNSUPPORTED"
    assert call(fkp, other) == invalid        # grids differ
    assert call(fkp, fkp) == invalid          # two f-k plans
    assert call(pfp, fkp) == invalid          # plans swapped
    assert call(fkp, half) == unsupported     # 16-bit storage
    nlos.reconstruct_moe(fkp, pfp, x, vf, vp)
    torch.cuda.synchronize()
    assert float(vf.abs().max()) == 0.0 and float(vp.abs().max()) == 0.0
