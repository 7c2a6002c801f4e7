"""Reduced-precision storage (FP16 / BF16 input and intermediates with a
per-volume scale, FP32 arithmetic) against the FP64 oracle run on the same
rounded input. FP16 must stay within relative L2 <= 2e-3 with the same peak
voxel; BF16 (8-bit mantissa) is reported and only held to a sanity bound."""
import numpy as np
import pytest

from oracle import fk, pf
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


def _fk(cap, storage):
    from paper_2608_28183_gb300 import nlos
    g = cap.geometry
    plan = nlos.plan_for_capture(g, "fk", storage)
    dt = plan.input_dtype()
    got = plan.reconstruct(to_device(cap.counts, dt)).cpu().numpy().astype(np.float64)
    ref = fk.fk_reconstruct(exact_input(cap.counts, dt), g.bin_width_s, g.wall_w_m, g.wall_h_m)
    return got, ref


@pytest.mark.parametrize("storage,tol", [("f16", 2e-3), ("bf16", 3e-2)])
def test_fk_reduced_precision_32x32x256(storage, tol):
    got, ref = _fk(synth.make_capture("fk_32x32x256", 0), storage)
    err = rel_l2(got, ref)
    print(f"f-k {storage} rel L2 {err:.3e}")
    assert err <= tol
    if storage == "f16":
        assert same_peak(got, ref, rtol=2e-3)


def test_fk_fp16_full_size_256x256x512():
    got, ref = _fk(synth.make_capture("fk_256x256x512", 0, device="cuda"), "f16")
    err = rel_l2(got, ref)
    print(f"f-k f16 256x256x512 rel L2 {err:.3e}")
    assert err <= 2e-3
    assert same_peak(got, ref, rtol=2e-3)


@pytest.mark.parametrize("storage,tol", [("f16", 2e-3), ("bf16", 3e-2)])
def test_pf_reduced_precision(storage, tol):
    from paper_2608_28183_gb300 import nlos
    g = synth.Geometry(32, 32, 512, 16e-12, 1.0, 1.0)
    rng = np.random.default_rng(4)
    pts = np.array([(rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), rng.uniform(0.5, 1.1), 1.0) for _ in range(3)])
    cap = synth.render(g, synth.Scene(points=pts), peak=400.0, background=0.5, seed=4)
    plan = nlos.plan_for_capture(g, "pf", storage, n_depths=40, depth_min_m=0.4, depth_max_m=1.2)
    dt = plan.input_dtype()
    got = plan.reconstruct(to_device(cap.counts, dt)).cpu().numpy().astype(np.float64)
    op = pf.make_plan(32, 32, 512, 16e-12, 1.0, 1.0, 40, 0.4, 1.2)
    ref = pf.pf_reconstruct(exact_input(cap.counts, dt), op)
    err = rel_l2(got, ref)
    print(f"pf {storage} rel L2 {err:.3e}")
    assert err <= tol
    if storage == "f16":
        assert same_peak(got, ref, rtol=2e-3)


def test_pf_fp16_workload_128x128x1024():
    from paper_2608_28183_gb300 import nlos
    cap = synth.make_capture("pf_128x128x1024", 0, device="cuda")
    g = cap.geometry
    plan = nlos.plan_for_capture(g, "pf", "f16", n_depths=128, depth_min_m=0.5, depth_max_m=2.5)
    got = plan.reconstruct(to_device(cap.counts, torch.float16)).cpu().numpy().astype(np.float64)
    op = pf.make_plan(128, 128, 1024, 16e-12, 2.0, 2.0, 128, 0.5, 2.5)
    ref = pf.pf_reconstruct(exact_input(cap.counts, torch.float16), op)
    err = rel_l2(got, ref)
    print(f"pf f16 128x128x1024 rel L2 {err:.3e}")
    assert err <= 2e-3
    assert same_peak(got, ref, rtol=2e-3)


@pytest.mark.parametrize("depths", [40, 7, 150])
def test_pf_fp16_tensor_core_and_ffma_depth_sums(depths):
    """FP16 phasor-field plans run the depth sum on the tensor cores (launch
    shape 0: persistent warp-specialised CTAs; shape 2: one CTA per tile) or
    on FP32 FMAs (shape 1): all within 2e-3 of the oracle and of each other,
    for depth counts below, inside and across the 128-depth blocks of the
    tensor-core forms."""
    from paper_2608_28183_gb300 import nlos
    g = synth.Geometry(32, 32, 512, 16e-12, 1.0, 1.0)
    rng = np.random.default_rng(depths)
    pts = np.array([(rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), rng.uniform(0.5, 1.1), 1.0) for _ in range(3)])
    cap = synth.render(g, synth.Scene(points=pts), peak=400.0, background=0.5, seed=depths)
    plan = nlos.plan_for_capture(g, "pf", "f16", n_depths=depths, depth_min_m=0.4, depth_max_m=1.2)
    names = [nlos.load_library().nlos_plan_stage_name(plan.handle, i).decode() for i in range(len(plan.tiles))]
    stage = names.index("pf_depth_sum")
    x = to_device(cap.counts, torch.float16)
    out = {}
    for v in (0, 1, 2):
        t = plan.tiles
        t[stage] = v
        plan.tiles = t
        out[v] = plan.reconstruct(x).cpu().numpy().astype(np.float64)
    op = pf.make_plan(32, 32, 512, 16e-12, 1.0, 1.0, depths, 0.4, 1.2)
    ref = pf.pf_reconstruct(exact_input(cap.counts, torch.float16), op)
    for v in (0, 1, 2):
        assert rel_l2(out[v], ref) <= 2e-3, (v, rel_l2(out[v], ref))
        assert same_peak(out[v], ref, rtol=2e-3)
    assert rel_l2(out[0], out[1]) <= 2e-3
    # the persistent form adds the parts of split tail tiles with f16 atomics
    assert rel_l2(out[2], out[0]) <= 1e-3


@pytest.mark.parametrize("storage,output,tol", [("f16", "magnitude", 2e-3), ("f16", "complex", 2e-3),
                                                ("bf16", "magnitude", 3e-2)])
def test_fk_reduced_precision_inverse_temporal_last(storage, output, tol):
    """A fused 64 x 64 x 256 plan takes the inverse temporal transform last in
    16-bit storage too (the kept spectrum stored in the storage type with its
    pass scale, the volume scale applied by the last stage)."""
    from paper_2608_28183_gb300 import nlos
    g = synth.Geometry(64, 64, 256, 32e-12, 1.0, 1.0)
    plan = nlos.plan_for_capture(g, "fk", storage, output=output)
    names = [nlos.load_library().nlos_plan_stage_name(plan.handle, i).decode() for i in range(len(plan.tiles))]
    assert "fk_z_inverse" in names
    cap = synth.make_capture("fk_32x32x256", 0, geom=g)
    dt = plan.input_dtype()
    got = plan.reconstruct(to_device(cap.counts, dt)).cpu().numpy()
    cpx = output == "complex"
    ref = fk.fk_reconstruct(exact_input(cap.counts, dt), g.bin_width_s, g.wall_w_m, g.wall_h_m, return_complex=cpx)
    err = rel_l2(got.astype(np.complex128 if cpx else np.float64), ref)
    print(f"f-k {storage} {output} 64x64x256 rel L2 {err:.3e}")
    assert err <= tol
    if storage == "f16":
        assert same_peak(np.abs(got), np.abs(ref), rtol=2e-3)
