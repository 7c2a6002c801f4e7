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
