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


# Per-atom bound that goes with every rel-RMS parity check of the GPU tests:
# no single atom may be off by more than PER_ATOM x tol x the RMS magnitude of
# the reference (a handful of wrong atoms would pass a norm over all atoms).
PER_ATOM = 10.0


def per_atom_worst(x, ref):
    """Largest per-atom error (Euclidean over the last axis of [N,3] arrays)
    over the RMS per-atom magnitude of ref, and that atom's index."""
    import numpy as np
    x, ref = np.asarray(x, float), np.asarray(ref, float)
    d = x - ref
    if d.ndim == 2:
        e = np.sqrt((d ** 2).sum(1))
        m = np.sqrt((ref ** 2).sum(1))
    else:
        e, m = np.abs(d), np.abs(ref)
    scale = float(np.sqrt((m ** 2).mean())) if m.size else 0.0
    if e.size == 0:
        return 0.0, -1
    i = int(np.argmax(e))
    return (float(e[i]) / scale if scale > 0 else float(e[i])), i


def assert_atoms(x, ref, tol, what=""):
    """rel-RMS(x, ref) <= tol and every atom within PER_ATOM * tol (relative
    to the RMS magnitude of ref)."""
    r = rel_rms(x, ref)
    assert r <= tol, ("rel-RMS", what, r, tol)
    w, i = per_atom_worst(x, ref)
    assert w <= PER_ATOM * tol, ("worst atom", what, i, w, PER_ATOM * tol)
