"""Failure detection without a GPU fault: a bounded device wait that nothing
satisfies gives up at its iteration limit and reports a timeout through the
error word, the context stays usable, and normal runs leave the word clear."""
import ctypes

import numpy as np
import pytest

from paper_2608_28183_gb300 import synth
from tests.gpu_util import to_device

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    from paper_2608_28183_gb300 import build, nlos
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return nlos.load_library()


def test_bounded_wait_times_out_and_context_survives(lib):
    from paper_2608_28183_gb300 import nlos
    code = ctypes.c_int(-1)
    st = lib.nlos_selftest_bounded_wait(2000, ctypes.byref(code))
    assert st == 5 and code.value == 1          # NLOS_ERR_TIMEOUT, timeout code
    g = synth.Geometry(32, 32, 256, 32e-12, 1.0, 1.0)
    plan = nlos.plan_for_capture(g, "fk", "f32")
    cap = synth.point_capture(g, [(0.1, 0.1, 0.6, 1.0)], peak=100.0)
    out = plan.reconstruct(to_device(cap.counts, torch.float32))
    torch.cuda.synchronize()
    assert torch.isfinite(out).all() and out.max() > 0
    code = ctypes.c_int(-1)
    assert lib.nlos_workspace_check(plan.handle, None, ctypes.byref(code)) == 0 and code.value == 0


def test_tma_staged_variants_leave_error_word_clear(lib):
    from paper_2608_28183_gb300 import nlos
    g = synth.Geometry(64, 64, 512, 16e-12, 1.0, 1.0)
    plan = nlos.plan_for_capture(g, "fk", "f32")
    cap = synth.make_capture("fk_32x32x256", 0, geom=g)
    x = to_device(cap.counts, torch.float32)
    base = plan.reconstruct(x).clone()
    n = len(plan.tiles)
    for stage in range(n):
        for v in (2, 3, 4, 5):
            tiles = [0] * n
            tiles[stage] = v
            try:
                plan.tiles = tiles
            except Exception:
                continue
            got = plan.reconstruct(x)
            err = float(torch.linalg.vector_norm((got - base).double()) / torch.linalg.vector_norm(base.double()))
            assert err <= 1e-6, (stage, v, err)
    code = ctypes.c_int(-1)
    assert lib.nlos_workspace_check(plan.handle, None, ctypes.byref(code)) == 0 and code.value == 0


def test_injected_allocation_failures_are_reported_and_leak_nothing(lib):
    """Host-side fault injection: each of the first allocations of a plan
    fails in turn; creation returns OUT_OF_MEMORY, releases what it had, and
    the next creation succeeds."""
    import ctypes
    from paper_2608_28183_gb300 import nlos
    g = synth.Geometry(32, 32, 256, 24e-12, 0.8, 0.8)
    desc = nlos.desc_for_capture(g, "pf", n_depths=16, depth_min_m=0.4, depth_max_m=1.0)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in range(1, 8):
        lib.nlos_debug_fail_allocation(k)
        h = ctypes.c_void_p()
        st = lib.nlos_plan_create(ctypes.byref(desc), ctypes.byref(h))
        lib.nlos_debug_fail_allocation(0)
        assert st == 2 and not h.value, (k, st)
        assert b"injected" in lib.nlos_last_error()
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (64 << 20)
    plan = nlos.plan_for_capture(g, "pf", n_depths=16, depth_min_m=0.4, depth_max_m=1.0)
    # a failure of the host-call staging leaves the plan usable
    x = torch.zeros((g.nx, g.ny, g.nt))
    v = torch.empty(plan.out_shape)
    lib.nlos_debug_fail_allocation(1)
    with pytest.raises(nlos.NlosError, match="OUT_OF_MEMORY"):
        plan.reconstruct_host(x, v)
    lib.nlos_debug_fail_allocation(0)
    plan.reconstruct_host(x, v)
    assert float(v.abs().sum()) == 0.0


def test_server_wait_times_out_then_completes(lib):
    from paper_2608_28183_gb300 import nlos
    g = synth.Geometry(128, 128, 512, 16e-12, 2.0, 2.0)
    server = nlos.Server(memory_budget_bytes=8 << 30, n_slots=2)
    desc = nlos.desc_for_capture(g, "fk")          # not preloaded: the plan is built on admission
    x = torch.zeros((g.nx, g.ny, g.nt), device="cuda")
    out = torch.empty((g.nx, g.ny, g.nt), device="cuda")
    t = server.submit(desc, x, out)
    with pytest.raises(nlos.NlosError, match="TIMEOUT"):
        server.wait(t, timeout_s=1e-4)
    assert server.wait(t, timeout_s=60.0) > 0
    torch.cuda.synchronize()
    assert float(out.abs().sum()) == 0.0


def test_bounds_check_records_without_access():
    """The bounds checks record an index outside its buffer (code 3) in the
    bounds-checked build and compile away in the normal one; the probe never
    touches memory outside the buffer either way."""
    import ctypes
    from paper_2608_28183_gb300 import build, nlos
    lib = nlos.load_library()
    code = ctypes.c_int(-1)
    assert lib.nlos_selftest_bounds(ctypes.byref(code)) == 0
    assert code.value == (3 if build.bounds_checked() else 0)
    assert (b"bounds-checked" in lib.nlos_version()) == build.bounds_checked()
