"""The grid geometry the CUDA library computes on the host (msm_geometry: no
device call) against the oracle's independent geometry routine, over
periodic and open boxes, cubic and not, both basis orders, automatic and
fixed level counts: level count, spacing, first index and extent of every
level.  No GPU needed."""
import ctypes as C

import numpy as np
import pytest

CASES = [
    # box, periodic, cutoff, spacing, levels, order
    ((62.2, 62.2, 62.2), True, 10.0, 2.0, 0, 3),     # the 23,558-atom box
    ((216.8, 216.8, 216.8), True, 12.0, 2.5, 0, 5),  # the 1.07M-atom box
    ((340.0, 340.0, 340.0), True, 10.0, 1.5, 5, 5),  # the 4.1M-atom box, l = 5
    ((30.0, 30.0, 30.0), False, 12.0, 2.5, 0, 3),    # the open 3,000-atom box
    ((24.0, 31.0, 40.0), True, 8.0, 1.7, 0, 3),      # not cubic
    ((24.0, 31.0, 40.0), False, 7.0, 1.7, 0, 5),
    ((40.0, 40.0, 40.0), True, 9.0, 2.0, 2, 3),      # fixed level counts
    ((40.0, 40.0, 40.0), False, 9.0, 2.0, 1, 5),
    ((20.0, 20.0, 20.0), True, 6.0, 2.0, 0, 5),
]


@pytest.fixture(scope="module")
def lib():
    from paper_1402_7216_gb300 import _capi, build
    return _capi.load(build.build())


@pytest.mark.parametrize("case", CASES, ids=[str(i) for i in range(len(CASES))])
def test_library_geometry_matches_oracle(case, lib, oracle):
    from paper_1402_7216_gb300._capi import MSMParams
    box, periodic, a, h, levels, order = case
    p = MSMParams()
    for d in range(3):
        p.box[d] = box[d]
    p.periodic, p.cutoff, p.spacing, p.levels, p.order = int(periodic), a, h, levels, order
    p.splitting, p.precision, p.coulomb_k, p.max_atoms = 2, 1, 1.0, 1000
    heff = (C.c_double * 3)()
    nlev = C.c_int(0)
    dims = (C.c_int * 48)()
    lo = (C.c_int * 48)()
    assert lib.msm_geometry(C.byref(p), heff, C.byref(nlev), dims, lo) == 0
    G = oracle.geometry(oracle.Params(box=box, periodic=periodic, cutoff=a, spacing=h, levels=levels, order=order))
    assert nlev.value == G.levels
    np.testing.assert_allclose(list(heff), G.h, rtol=1e-15)
    for k in range(G.levels):
        assert tuple(dims[3 * k:3 * k + 3]) == tuple(G.n[k]), k
        assert tuple(lo[3 * k:3 * k + 3]) == tuple(G.lo[k]), k


def test_geometry_rejects_what_msm_create_rejects(lib):
    from paper_1402_7216_gb300._capi import MSMParams
    p = MSMParams()
    for d in range(3):
        p.box[d] = 20.0
    p.periodic, p.cutoff, p.spacing, p.levels, p.order = 1, 12.0, 2.0, 0, 3   # a > L/2
    p.splitting, p.precision, p.coulomb_k, p.max_atoms = 2, 1, 1.0, 10
    assert lib.msm_geometry(C.byref(p), None, None, None, None) == -3
    p.cutoff, p.order = 6.0, 4                                             # no such basis
    assert lib.msm_geometry(C.byref(p), None, None, None, None) == -1
    assert lib.msm_geometry(None, None, None, None, None) == -1
