import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def rel_err(got, ref):
    """Componentwise |g - o| / max(|o|, ||o||_inf of that vector, 1e-300) (max over all)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.maximum(np.abs(ref), np.max(np.abs(ref), axis=-1, keepdims=True))
    scale = np.maximum(scale, 1e-300)
    return float(np.max(np.abs(got - ref) / scale))


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle
