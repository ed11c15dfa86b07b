"""Autotuned tile shapes: the search returns a candidate of its own space, the
tuned plan gives the default plan's results (tile shapes only change the
summation order), and the cache answers the second request."""
import numpy as np
import pytest
import torch

from conftest import rel_rms
from synth import make_water_box

pytestmark = pytest.mark.gpu


def test_autotune_search_result_and_cache(tmp_path, monkeypatch):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_7216_gb300 import MSM
    from paper_1402_7216_gb300 import autotune as AT
    monkeypatch.setenv("MSM_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    dev = torch.device("cuda:0")
    pos_h, q_h = make_water_box(40.0, 2000, 4, 4, seed=51, periodic=True)
    pos, q = torch.tensor(pos_h, device=dev), torch.tensor(q_h, device=dev)
    kw = dict(box=40.0, periodic=True, cutoff=9.0, spacing=2.0, order=5, splitting=2, precision="mixed")
    tuning, times = AT.autotune(pos, q, reps=3, **kw)
    space = dict(AT.SEARCH)
    for k, v in tuning.items():
        assert v in space[k]
    assert "default" in times and len(times) > 3
    t2, times2 = AT.autotune(pos, q, reps=3, **kw)
    assert t2 == tuning and "cached" in times2
    base = MSM(max_atoms=len(q_h), **kw)
    for t in [tuning, {"cell_fill": 40, "patch_cells": 2, "lattice_waves": 8}]:
        tuned = MSM(max_atoms=len(q_h), tuning=t, **kw)
        E0, phi0, F0 = base.eval(pos, q)
        E1, phi1, F1 = tuned.eval(pos, q)
        torch.cuda.synchronize()
        assert abs(E1.item() - E0.item()) <= 1e-6 * abs(E0.item())
        assert rel_rms(F1.cpu().numpy(), F0.cpu().numpy()) <= 1e-5
        assert rel_rms(phi1.cpu().numpy(), phi0.cpu().numpy()) <= 1e-6


def test_tuning_fields_are_checked():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_7216_gb300 import MSM, MSMError
    with pytest.raises(MSMError):
        MSM(box=30.0, periodic=True, cutoff=9.0, spacing=2.0, max_atoms=100, tuning={"patch_cells": 7})
