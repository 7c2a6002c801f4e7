"""The C-ABI library loads and exports every function include/nlos.h declares;
argument validation happens on the host before any device work (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2608_28183_gb300 import build as nbuild
from paper_2608_28183_gb300 import nlos

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    nbuild.build()
    return nlos.load_library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "nlos.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nlos_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(nlos.EXPORTED)


def test_version_and_defaults(lib):
    assert b"sm_103a" in lib.nlos_version()
    d = nlos.PlanDesc()
    lib.nlos_plan_desc_default(ctypes.byref(d))
    assert (d.method, d.storage, d.pad_factor, d.cycles) == (0, 0, 2, 5.0)


def _create(lib, **kw):
    d = nlos.PlanDesc()
    lib.nlos_plan_desc_default(ctypes.byref(d))
    d.nx, d.ny, d.nt, d.bin_width_s, d.wall_w_m, d.wall_h_m = 32, 32, 256, 32e-12, 1.0, 1.0
    for k, v in kw.items():
        setattr(d, k, v)
    h = ctypes.c_void_p()
    st = lib.nlos_plan_create(ctypes.byref(d), ctypes.byref(h))
    return st, lib.nlos_last_error().decode()


@pytest.mark.parametrize("kw,status", [
    (dict(nx=0), 1), (dict(bin_width_s=0.0), 1), (dict(wall_w_m=-1.0), 1), (dict(method=7), 1),
    (dict(storage=9), 1), (dict(pad_factor=3), 1), (dict(pad_factor=1, method=1, n_depths=8,
                                                           depth_min_m=0.5, depth_max_m=1.0), 4),
    (dict(pad_factor=1, nx=8), 4), (dict(pad_factor=1, nx=24), 4), (dict(nt=8192), 4), (dict(nx=2048), 4),
    (dict(nx=4, ny=4), 4), (dict(method=1, n_depths=0), 1),
    (dict(method=1, n_depths=8, depth_min_m=1.0, depth_max_m=0.5), 1), (dict(output=2), 1), (dict(output=-1), 1),
    (dict(method=2, storage=1, n_depths=8, depth_min_m=0.5, depth_max_m=1.0), 4),
    (dict(method=1, n_depths=8, depth_min_m=0.5, depth_max_m=1.0, sigma_s=0, sigma_t=1), 1),
    (dict(method=1, n_depths=8, depth_min_m=0.5, depth_max_m=1.0, wavelength_m=-0.01), 1),
])
def test_invalid_descriptions_rejected_before_device_work(lib, kw, status):
    st, msg = _create(lib, **kw)
    assert st == status and msg


def test_null_arguments(lib):
    assert lib.nlos_plan_create(None, None) == 1
    assert lib.nlos_reconstruct(None, None, None, None) == 1
    assert lib.nlos_plan_query(None, None, None, None, None) == 1
    assert lib.nlos_plan_destroy(None) == 1
    assert lib.nlos_max_image(None, 4, 4, 4, 0, None, None) == 1
    assert lib.nlos_moe_mix(None, None, 10, 0.3, 1e-3, None, None) == 1
    assert lib.nlos_coherence_merge(None, 2, 10, 1e-6, None, None, None) == 1
    assert lib.nlos_dda(None, 2, 10, 4, None, None) == 1
    assert lib.nlos_bin_transient(None, None, 10, 4, 4, 16, 0, 1, 0, None, None) == 1
    assert lib.nlos_bin_phasors(None, None, None, 10, 0, 1, 0, None, None) == 1
    assert lib.nlos_plan_band(None, None, None) == 1
    assert lib.nlos_reconstruct_phasors(None, None, None, None) == 1
    assert lib.nlos_reconstruct_host_many(None, None, None, 1, None) == 1
    assert lib.nlos_reconstruct_batch(None, None, None, None, -1, None) == 1
    assert lib.nlos_reconstruct_batch(None, None, None, None, 0, None) == 0
    assert lib.nlos_ffma_rate_launch(None, None, 1, 1, None, None) == 1


def test_binding_rejects_host_tensors_before_device_work(lib):
    """The Python binding only marshals: tensors that are not contiguous CUDA
    tensors of the right type are refused before any library call, and there
    is no host fallback to take them instead."""
    torch = pytest.importorskip("torch")
    v = torch.zeros((4, 4, 8), dtype=torch.float32)
    with pytest.raises(ValueError, match="CUDA"):
        nlos.max_image(v)
    with pytest.raises(ValueError, match="CUDA"):
        nlos.moe_mix(v[0], v[1])
    with pytest.raises(ValueError, match="CUDA"):
        nlos.dda([v, v])
    px = torch.zeros(16, dtype=torch.int32)
    with pytest.raises(ValueError, match="uint32"):
        nlos.bin_transient(px, px, 4, 4, 8, 0, 1)
