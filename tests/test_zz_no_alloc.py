"""nlos_reconstruct_noalloc: the reconstruction entry point that allocates nothing.

It is for callers that cannot call cudaMalloc while they reconstruct
(real-time loops, where an allocation may stall a frame; applications that
give the library a fixed share of device memory and pool the rest
themselves): it runs an existing plan with its scratch in a fixed 32 MiB
device array held by the library. Its output must match nlos_reconstruct's (the entry point that
uses the plan's own workspace) within the parity tolerance, on two calls in a
row (the array keeps the previous call's contents, so the second call checks
that nothing stale leaks in). This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2608_28183_gb300 import synth
from tests.gpu_util import rel_l2, to_device

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    from paper_2608_28183_gb300 import build, nlos
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return nlos.load_library()


def _noalloc(lib, plan, H, out):
    st = lib.nlos_reconstruct_noalloc(plan.handle, ctypes.c_void_p(H.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.nlos_last_error().decode()


def _check_two_calls(lib, plan, inputs):
    for H in inputs:
        ref = plan.reconstruct(H)                  # plan's own workspace
        out = torch.full(plan.out_shape, float("nan"), device="cuda")
        _noalloc(lib, plan, H, out)
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_l2(got, want) <= 1e-5


def test_noalloc_fk_matches_workspace_path(lib):
    from paper_2608_28183_gb300 import nlos
    cap0 = synth.make_capture("fk_32x32x256", 0)
    cap1 = synth.make_capture("fk_32x32x256", 1)
    plan = nlos.plan_for_capture(cap0.geometry, "fk", "f32")
    assert plan.workspace_bytes <= 32 << 20
    _check_two_calls(lib, plan, [to_device(cap0.counts, torch.float32), to_device(cap1.counts, torch.float32)])


def test_noalloc_phasor_matches_workspace_path(lib):
    from paper_2608_28183_gb300 import nlos
    g = synth.Geometry(32, 32, 512, 16e-12, 1.0, 1.0)
    plan = nlos.plan_for_capture(g, "pf", "f32", n_depths=40, depth_min_m=0.4, depth_max_m=1.2)
    caps = [synth.point_capture(g, [(0.1 * k, -0.1, 0.7 + 0.1 * k, 1.0)], peak=300.0, background=0.5,
                                seed=k, noise=True) for k in range(2)]
    _check_two_calls(lib, plan, [to_device(c.counts, torch.float32) for c in caps])


def test_noalloc_rejects_plans_beyond_its_scratch(lib):
    from paper_2608_28183_gb300 import nlos
    plan = nlos.Plan(128, 128, 256, 16e-12, 2.0, 2.0, "fk", "f32")
    assert plan.workspace_bytes > 32 << 20
    H = torch.zeros((128, 128, 256), dtype=torch.float32, device="cuda")
    out = plan.empty_volume()
    st = lib.nlos_reconstruct_noalloc(plan.handle, ctypes.c_void_p(H.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 1 and b"scratch" in lib.nlos_last_error()
