import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(autouse=True)
def _workspace_error_words():
    """In the bounds-checked build (NLOS_BOUNDS_CHECK=1) every plan a test
    closed must have left its device error word at 0."""
    yield
    if os.environ.get("NLOS_BOUNDS_CHECK", "0") in ("", "0"):
        return
    import gc
    from paper_2608_28183_gb300 import nlos
    gc.collect()
    errors = list(nlos.WORKSPACE_ERRORS)
    nlos.WORKSPACE_ERRORS.clear()
    assert not errors, f"device error words set: {errors}"
