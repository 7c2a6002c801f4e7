"""GPU parity of f-k migration through the C ABI against the FP64 oracle.

FP32 storage must match to relative L2 <= 1e-5 with identical peak voxels
(the oracle runs on the same inputs, converted exactly to float64).
"""
import math

import numpy as np
import pytest

from oracle import fk
from paper_2608_28183_gb300 import synth
from tests.gpu_util import exact_input, local_peaks_agree, rel_l2, same_peak, to_device

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def library():
    from paper_2608_28183_gb300 import build, nlos
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return nlos.load_library()


def _plan(geom, storage="f32"):
    from paper_2608_28183_gb300 import nlos
    return nlos.plan_for_capture(geom, "fk", storage)


def _gpu(plan, H, dtype=None):
    dtype = dtype or plan.input_dtype()
    out = plan.reconstruct(to_device(H, dtype))
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def _oracle(geom, H):
    return fk.fk_reconstruct(H, geom.bin_width_s, geom.wall_w_m, geom.wall_h_m)


def _noise_capture(geom, seed):
    rng = np.random.default_rng(seed)
    pts = [(rng.uniform(-0.3, 0.3) * geom.wall_w_m, rng.uniform(-0.3, 0.3) * geom.wall_h_m,
            rng.uniform(0.3, 0.8) * geom.nt * geom.bin_depth_m, 1.0) for _ in range(2)]
    return synth.render(geom, synth.Scene(points=np.array(pts)), peak=200.0, background=0.5, seed=seed)


SMALL = [
    synth.Geometry(8, 8, 16, 300e-12, 0.3, 0.3),          # minimum sizes
    synth.Geometry(8, 16, 64, 64e-12, 0.4, 0.9),          # non-square, several tiles along y
    synth.Geometry(16, 32, 128, 32e-12, 0.8, 1.3),
    synth.Geometry(64, 8, 32, 100e-12, 1.5, 0.3),         # long x, short t
    synth.Geometry(32, 32, 512, 16e-12, 1.0, 1.0),
]


@pytest.mark.parametrize("geom", SMALL, ids=lambda g: f"{g.nx}x{g.ny}x{g.nt}")
def test_fk_parity_small(geom):
    cap = _noise_capture(geom, seed=geom.nx * 7 + geom.nt)
    plan = _plan(geom)
    got = _gpu(plan, cap.counts)
    ref = _oracle(geom, exact_input(cap.counts, torch.float32))
    assert rel_l2(got, ref) <= 1e-5
    assert same_peak(got, ref)


def test_fk_parity_workload_32x32x256():
    cap = synth.make_capture("fk_32x32x256", 0)
    g = cap.geometry
    plan = _plan(g)
    got = _gpu(plan, cap.counts)
    ref = _oracle(g, exact_input(cap.counts, torch.float32))
    err = rel_l2(got, ref)
    assert err <= 1e-5, err
    assert same_peak(got, ref)
    xs, ys = synth.wall_coords(g.nx, g.wall_w_m), synth.wall_coords(g.ny, g.wall_h_m)
    centres = [(np.argmin(abs(xs - p[0])), np.argmin(abs(ys - p[1])), math.floor(p[2] / g.bin_depth_m))
               for p in cap.scene.points]
    assert local_peaks_agree(got, ref, centres)


def test_fk_parity_full_size_256x256x512():
    """Full-size workload in the benchmark's launch configuration."""
    cap = synth.make_capture("fk_256x256x512", 0, device="cuda")
    g = cap.geometry
    plan = _plan(g)
    got = _gpu(plan, cap.counts)
    ref = _oracle(g, exact_input(cap.counts, torch.float32))
    err = rel_l2(got, ref)
    assert err <= 1e-5, err
    assert same_peak(got, ref)
    centres = [(np.argmin(abs(synth.wall_coords(g.nx, g.wall_w_m) - p[0])),
                np.argmin(abs(synth.wall_coords(g.ny, g.wall_h_m) - p[1])),
                math.floor(p[2] / g.bin_depth_m)) for p in cap.scene.points]
    assert local_peaks_agree(got, ref, centres)


def test_fk_zero_input_gives_zero_volume():
    g = SMALL[2]
    plan = _plan(g)
    got = _gpu(plan, np.zeros((g.nx, g.ny, g.nt)))
    assert np.all(got == 0.0)


def test_fk_deterministic_and_host_path():
    g = SMALL[4]
    cap = _noise_capture(g, seed=3)
    plan = _plan(g)
    a = _gpu(plan, cap.counts)
    b = _gpu(plan, cap.counts)
    assert np.array_equal(a, b)
    h_in = torch.as_tensor(cap.counts, dtype=torch.float32).contiguous().pin_memory()
    h_out = torch.empty(plan.out_shape, dtype=torch.float32).pin_memory()
    plan.reconstruct_host(h_in, h_out)
    assert np.array_equal(h_out.numpy().astype(np.float64), a)


@pytest.mark.parametrize("n", [1, 2, 7])
def test_fk_pipelined_host_calls(n):
    """n captures host -> host through the pipelined entry point equal the
    device path capture by capture (more captures than staging slots, and
    pageable as well as page-locked host memory)."""
    g = SMALL[4]
    plan = _plan(g)
    caps = [_noise_capture(g, seed=10 + i).counts for i in range(n)]
    ins = [torch.as_tensor(c, dtype=torch.float32).contiguous() for c in caps]
    if n != 2:
        ins = [t.pin_memory() for t in ins]
    outs = [torch.full(plan.out_shape, -1.0, dtype=torch.float32) for _ in range(n)]
    plan.reconstruct_host_many(ins, outs)
    for c, o in zip(caps, outs):
        assert np.array_equal(o.numpy().astype(np.float64), _gpu(plan, c))
    # the plan stays usable for other calls, and a second pipelined call reuses the staging
    plan.reconstruct_host_many(ins[:1], outs[:1])
    assert np.array_equal(outs[0].numpy().astype(np.float64), _gpu(plan, caps[0]))


def test_fk_batch_matches_single_calls():
    from paper_2608_28183_gb300 import nlos
    geoms = [SMALL[1], SMALL[2], SMALL[4], SMALL[2]]
    plans = [_plan(g) for g in geoms[:3]]
    plans.append(plans[1])                        # same plan twice -> explicit workspaces
    caps = [_noise_capture(g, seed=11 + i) for i, g in enumerate(geoms)]
    ins = [to_device(c.counts, torch.float32) for c in caps]
    outs = [p.empty_volume() for p in plans]
    wss = [torch.empty(p.workspace_bytes, dtype=torch.uint8, device="cuda") for p in plans]
    nlos.reconstruct_batch(plans, ins, outs, wss)
    torch.cuda.synchronize()
    for p, c, o in zip(plans, caps, outs):
        assert np.array_equal(o.cpu().numpy().astype(np.float64), _gpu(p, c.counts))


UNPADDED = [
    synth.Geometry(16, 16, 16, 300e-12, 0.5, 0.5),        # minimum unpadded sizes
    synth.Geometry(32, 16, 128, 32e-12, 1.0, 0.6),        # non-square
    synth.Geometry(64, 64, 512, 16e-12, 1.5, 1.5),
]


@pytest.mark.parametrize("geom", UNPADDED, ids=lambda g: f"{g.nx}x{g.ny}x{g.nt}")
def test_fk_unpadded_parity(geom):
    """The unpadded variant (Pad x1) against the oracle with pad_factor 1."""
    from paper_2608_28183_gb300 import nlos
    cap = _noise_capture(geom, seed=geom.nx + 3 * geom.nt)
    plan = nlos.plan_for_capture(geom, "fk", "f32", pad_factor=1)
    got = _gpu(plan, cap.counts)
    ref = fk.fk_reconstruct(exact_input(cap.counts, torch.float32), geom.bin_width_s, geom.wall_w_m,
                            geom.wall_h_m, pad_factor=1)
    assert rel_l2(got, ref) <= 1e-5
    assert same_peak(got, ref)


def test_fk_unpadded_fp16():
    from paper_2608_28183_gb300 import nlos
    geom = UNPADDED[2]
    cap = _noise_capture(geom, seed=9)
    plan = nlos.plan_for_capture(geom, "fk", "f16", pad_factor=1)
    got = _gpu(plan, cap.counts)
    ref = fk.fk_reconstruct(exact_input(cap.counts, torch.float16), geom.bin_width_s, geom.wall_w_m,
                            geom.wall_h_m, pad_factor=1)
    assert rel_l2(got, ref) <= 2e-3


ANY_SIZE = [
    synth.Geometry(24, 40, 200, 32e-12, 0.8, 1.3),       # every axis padded to the next power of two >= 2x
    synth.Geometry(20, 28, 300, 24e-12, 0.7, 0.9),
    synth.Geometry(96, 80, 300, 24e-12, 1.2, 1.0),
]


@pytest.mark.parametrize("geom", ANY_SIZE, ids=lambda g: f"{g.nx}x{g.ny}x{g.nt}")
def test_fk_parity_any_size(geom):
    """Grids with no power-of-two axis against the oracle with the same padding."""
    cap = _noise_capture(geom, seed=geom.nt)
    plan = _plan(geom)
    got = _gpu(plan, cap.counts)
    ref = _oracle(geom, exact_input(cap.counts, torch.float32))
    assert rel_l2(got, ref) <= 1e-5
    assert same_peak(got, ref)


def test_fk_any_size_fp16():
    geom = ANY_SIZE[1]
    cap = _noise_capture(geom, seed=4)
    plan = _plan(geom, "f16")
    got = _gpu(plan, cap.counts)
    ref = _oracle(geom, exact_input(cap.counts, torch.float16))
    assert rel_l2(got, ref) <= 2e-3


FUSED = [
    (synth.Geometry(48, 64, 256, 32e-12, 1.0, 1.2), "f32", "magnitude"),     # L = 128, a not a power of two
    (synth.Geometry(64, 48, 160, 24e-12, 1.2, 0.9), "f32", "magnitude"),     # Lx = Ly = 128, b not a power of two
    (synth.Geometry(128, 128, 512, 16e-12, 2.0, 2.0), "f32", "magnitude"),   # L = 256
    (synth.Geometry(200, 256, 64, 32e-12, 1.6, 2.0), "f32", "magnitude"),    # L = 512, a not a power of two
    (synth.Geometry(64, 64, 256, 32e-12, 1.0, 1.0), "f32", "complex"),
    (synth.Geometry(128, 128, 256, 16e-12, 2.0, 2.0), "f16", "magnitude"),
]


@pytest.mark.parametrize("geom,storage,output", FUSED,
                         ids=lambda v: f"{v.nx}x{v.ny}x{v.nt}" if hasattr(v, "nx") else str(v))
def test_fk_fused_lateral_matches_separate(geom, storage, output):
    """The fused x/y forward and y/x inverse stages (one launch each, the
    intermediate kept in L2) give the volume of the four separate axis passes
    (same arithmetic; float32 to rounding), and their chunk waits never run
    out (device error word 0)."""
    import ctypes
    from paper_2608_28183_gb300 import nlos
    cap = _noise_capture(geom, seed=geom.nx + geom.nt)
    fused = nlos.plan_for_capture(geom, "fk", storage, output=output)
    sep = nlos.plan_for_capture(geom, "fk", storage, output=output, separate_axes=True)
    lib = nlos.load_library()
    names = [lib.nlos_plan_stage_name(fused.handle, i).decode() for i in range(len(fused.tiles))]
    assert "fk_xy_forward" in names and "fk_yx_inverse" in names
    x = to_device(cap.counts, fused.input_dtype())
    for _ in range(2):          # the second call reuses the counters cleared by the first
        a = fused.reconstruct(x)
    b = sep.reconstruct(x)
    torch.cuda.synchronize()
    code = ctypes.c_int(-1)
    assert lib.nlos_workspace_check(fused.handle, None, ctypes.byref(code)) == 0 and code.value == 0
    an, bn = a.cpu().numpy(), b.cpu().numpy()
    err = rel_l2(an, bn)
    assert err <= (1e-6 if storage == "f32" else 2e-3), err
    if storage == "f32" and output == "magnitude":
        ref = _oracle(geom, exact_input(cap.counts, torch.float32))
        assert rel_l2(an.astype(np.float64), ref) <= 1e-5
        assert same_peak(an, ref)
