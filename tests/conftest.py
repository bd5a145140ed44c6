import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Both native libraries are built before any test imports them (a no-op when the
# sources are unchanged); nvcc cross-compiles without a GPU.
import __graft_entry__  # noqa: E402

__graft_entry__._load_build_module().build()
import oracle  # noqa: E402

oracle.build()


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if cuda_available():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


# The FP32-mode bar of every phi comparison against the FP64 oracle:
# |gpu - oracle| <= 1e-6 + 1e-5 |oracle|, element by element.
PHI_ATOL, PHI_RTOL = 1e-6, 1e-5


def assert_phi_close(got, want, label=""):
    import numpy as np
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    assert got.shape == want.shape, (label, got.shape, want.shape)
    err = np.abs(got - want)
    bound = PHI_ATOL + PHI_RTOL * np.abs(want)
    bad = err > bound
    assert not bad.any(), (f"{label}: {int(bad.sum())} of {bad.size} entries off; worst excess "
                           f"{(err - bound).max():.3e}, max |err| {err.max():.3e}")
    return float(err.max()) if err.size else 0.0
