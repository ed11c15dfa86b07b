import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library through its C ABI)")


@pytest.fixture(scope="session")
def oracle():
    import oracle as O
    O.lib()
    return O


def rel_rms(x, ref):
    import numpy as np
    x, ref = np.asarray(x, float), np.asarray(ref, float)
    return float(np.sqrt(((x - ref) ** 2).sum() / (ref ** 2).sum()))
