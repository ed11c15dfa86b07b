"""msm_energy_noalloc: the energy reduction for callers that must not allocate
device memory (an engine whose pool owns all device memory, or a step loop
that cannot afford cudaMalloc).  Its scratch is a file-scope device array, so
the call allocates nothing; here it is checked through the C ABI against the
energy msm_eval returns for the same charges and potentials, on two calls in
a row (the second reuses the array the first one left behind)."""
import ctypes

import numpy as np
import pytest
import torch

from synth import make_water_box

pytestmark = pytest.mark.gpu


def test_energy_noalloc_matches_msm_eval_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_7216_gb300 import MSM, lib
    L = lib()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream()
    for seed, nw in [(31, 900), (32, 500)]:        # the second call is smaller than the first
        pos, q = make_water_box(30.0, nw, 2, 2, seed=seed, periodic=True)
        plan = MSM(box=30.0, periodic=True, cutoff=9.0, spacing=2.0, order=3, splitting=2,
                   precision="fp64", max_atoms=len(q))
        tq = torch.tensor(q, device=dev)
        E, phi, _ = plan.eval(torch.tensor(pos, device=dev), tq)
        out = torch.full((), float("nan"), dtype=torch.float64, device=dev)
        rc = L.msm_energy_noalloc(len(q), ctypes.c_void_p(tq.data_ptr()), ctypes.c_void_p(phi.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        assert np.isfinite(out.item())
        # FP64 on both sides; only the order of the final sums may differ
        assert abs(out.item() - E.item()) <= 1e-10 * abs(E.item())
        plan.close()
    # limits and arguments are checked before anything runs
    assert L.msm_energy_noalloc(256 * 65536 + 1, ctypes.c_void_p(tq.data_ptr()), ctypes.c_void_p(phi.data_ptr()),
                                ctypes.c_void_p(out.data_ptr()), None) == -9
    assert L.msm_energy_noalloc(4, None, None, ctypes.c_void_p(out.data_ptr()), None) == -1
