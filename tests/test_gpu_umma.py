"""Tensor-core (tcgen05) self-check: shared-memory descriptors, the kind::f16
instruction descriptor and tensor-memory reads give the exact product of
small-integer matrices."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    from paper_2608_28183_gb300 import build, nlos
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return nlos.load_library()


@pytest.mark.parametrize("n_cols", [16, 64, 256])
def test_umma_product_is_exact(lib, n_cols):
    r = np.arange(128)[:, None]
    n = np.arange(n_cols)[:, None]
    k = np.arange(64)[None, :]
    A = ((r * 3 + k * 5) % 7 - 3).astype(np.float64)
    B = ((n * 2 + k * 7) % 5 - 2).astype(np.float64)
    out = torch.full((128, n_cols), float("nan"), device="cuda")
    code = ctypes.c_int(-1)
    st = lib.nlos_selftest_umma(n_cols, ctypes.c_void_p(out.data_ptr()), ctypes.byref(code))
    assert st == 0 and code.value == 0, lib.nlos_last_error()
    np.testing.assert_array_equal(out.cpu().numpy().astype(np.float64), A @ B.T)


def test_ffma_rate_is_plausible(lib):
    """The FMA-chain probe runs and reports a rate between a tenth of and the
    nominal FP32 FMA peak of 152 SMs x 128 lanes x 2 flop x 2.07 GHz."""
    from paper_2608_28183_gb300 import nlos
    rate = nlos.ffma_rate(blocks=152 * 4, iters=256, repeats=2)
    assert 0.1 * 80.5 < rate < 1.02 * 80.5, rate
