"""CPU checks of the C ABI boundary: the CUDA library builds, loads and exports
every entry point include/msm.h declares (no compute calls: no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "msm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(msm_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def library():
    from paper_1402_7216_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ["msm_create", "msm_destroy", "msm_eval", "msm_eval_backward", "msm_eval_host",
              "msm_status", "msm_query", "msm_strerror"]:
        assert s in syms


def test_library_exports_every_declared_symbol(library):
    for s in declared_symbols():
        assert hasattr(library, s), s


def test_binding_names_match_header():
    from paper_1402_7216_gb300 import _capi
    assert sorted(_capi.EXPORTS) == sorted(declared_symbols())


def test_strerror_is_pure_host(library):
    library.msm_strerror.restype = ctypes.c_char_p
    assert library.msm_strerror(0) == b"ok"
    assert b"capacity" in library.msm_strerror(-9)
    assert library.msm_strerror(12345) == b"unknown error"


def test_create_rejects_bad_parameters_without_a_gpu(library):
    # parameter validation happens before any device call
    from paper_1402_7216_gb300 import _capi
    L = _capi.load()
    h = ctypes.c_void_p()
    p = _capi.MSMParams()
    for d in range(3):
        p.box[d] = 30.0
    p.periodic, p.cutoff, p.spacing, p.order, p.splitting = 1, 10.0, 2.0, 4, 2
    p.precision, p.coulomb_k, p.max_atoms = 1, 1.0, 100
    assert L.msm_create(ctypes.byref(p), ctypes.byref(h)) == -1        # order 4
    p.order = 3
    p.cutoff = 16.0
    assert L.msm_create(ctypes.byref(p), ctypes.byref(h)) == -3        # a > L/2
    p.cutoff = 13.0
    assert L.msm_create(ctypes.byref(p), ctypes.byref(h)) == -2        # fewer than 5 cells
    assert L.msm_create(None, ctypes.byref(h)) == -1


def test_create_tuned_rejects_bad_tuning_without_a_gpu(library):
    # the tuning ranges are checked on the host before any device call
    from paper_1402_7216_gb300 import _capi
    L = _capi.load()
    h = ctypes.c_void_p()
    p = _capi.MSMParams()
    for d in range(3):
        p.box[d] = 30.0
    p.periodic, p.cutoff, p.spacing, p.order, p.splitting = 1, 9.0, 2.0, 3, 2
    p.precision, p.coulomb_k, p.max_atoms = 1, 1.0, 100
    for bad in [(-1, 0, 0), (257, 0, 0), (0, 5, 0), (0, -2, 0), (0, 0, 65), (0, 0, -1)]:
        t = _capi.MSMTuning(*bad)
        assert L.msm_create_tuned(ctypes.byref(p), ctypes.byref(t), ctypes.byref(h)) == -1, bad
    for field, bad in [("pair_runs", 3), ("pair_runs", -1), ("pair_targets", 16), ("lattice_method", 3)]:
        t = _capi.MSMTuning()
        setattr(t, field, bad)
        assert L.msm_create_tuned(ctypes.byref(p), ctypes.byref(t), ctypes.byref(h)) == -1, (field, bad)
    p.order = 4  # bad params are still reported with a valid tuning
    t = _capi.MSMTuning(26, 4, 4)
    assert L.msm_create_tuned(ctypes.byref(p), ctypes.byref(t), ctypes.byref(h)) == -1
