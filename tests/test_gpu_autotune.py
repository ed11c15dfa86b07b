"""Autotuned tile shapes: the search returns a candidate of its own space, the
tuned plan gives the default plan's results (tile shapes only change the
summation order), and the cache answers the second request."""
import numpy as np
import pytest
import torch

from conftest import assert_atoms, rel_rms
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
    for k, v in times["choice"].items():
        assert tuple(v) in space[k] if k == "lattice_tile" else v in space[k]
    assert "default" in times and len(times) > 6
    assert any("lattice_method=1" in k for k in times)          # the stencil against the FFT default
    # the stencil's tiles are searched exactly when the stencil won
    assert any("lattice_tile=" in k for k in times) == AT.uses_stencil(times["choice"])
    assert any("pair_targets=8" in k for k in times)            # and the pair clusters
    t2, times2 = AT.autotune(pos, q, reps=3, **kw)
    assert t2 == tuning and "cached" in times2
    base = MSM(max_atoms=len(q_h), **kw)
    for t in [tuning, {"cell_fill": 40, "patch_cells": 2, "lattice_waves": 8, "lattice_method": 1},
              {"pair_targets": 8, "lattice_txn": 2, "lattice_tyn": 16, "lattice_method": 1}]:
        tuned = MSM(max_atoms=len(q_h), tuning=t, **kw)
        E0, phi0, F0 = base.eval(pos, q)
        E1, phi1, F1 = tuned.eval(pos, q)
        torch.cuda.synchronize()
        assert abs(E1.item() - E0.item()) <= 1e-6 * abs(E0.item())
        assert_atoms(F1.cpu().numpy(), F0.cpu().numpy(), 1e-5)
        assert_atoms(phi1.cpu().numpy(), phi0.cpu().numpy(), 1e-6)


def test_tuning_fields_are_checked():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_7216_gb300 import MSM, MSMError
    for bad in [{"patch_cells": 7}, {"pair_targets": 16}, {"lattice_txn": 4}, {"lattice_txn": 8, "lattice_tyn": 8},
                {"lattice_txn": 32, "lattice_tyn": 1}]:   # the last: a 343 x 80 window, too wide for shared memory
        with pytest.raises(MSMError) as e:
            MSM(box=30.0, periodic=True, cutoff=9.0, spacing=0.45, max_atoms=100, tuning=bad)
        assert e.value.code == -1, bad


def test_autotune_batch_search_and_cache(tmp_path, monkeypatch):
    """The batch tuner times the captured batch graph per candidate, returns
    a candidate of its search space, and answers the second request from
    the cache; a batch built with the chosen tuning gives the same results."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_7216_gb300 import MSM, MSMBatch
    from paper_1402_7216_gb300 import autotune as AT
    monkeypatch.setenv("MSM_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    dev = torch.device("cuda:0")
    boxes, ps, qs = [], [], []
    for i, nw in enumerate([500, 900, 700]):
        L = (3 * nw / 0.1) ** (1.0 / 3.0)
        p, qq = make_water_box(L, nw, 0, 0, seed=60 + i, periodic=True)
        boxes.append(L)
        ps.append(p)
        qs.append(qq)
    counts = [len(qq) for qq in qs]
    pos = torch.tensor(np.vstack(ps), device=dev)
    q = torch.tensor(np.concatenate(qs), device=dev)
    kw = dict(cutoff=6.0, spacing=1.5, order=3, splitting=2)
    tunings, summary, times = AT.autotune_batch(boxes, pos, q, counts, reps=2, **kw)
    space = dict(AT.SEARCH_BATCH)
    for k, v in summary["shared"].items():
        assert v in space[k]
    for g, tile in summary["lattice_tile_by_grid0"].items():
        assert int(g) in summary["grid0_sizes"] and tuple(tile) in AT.TILES_BATCH
    assert len(tunings) == len(counts)
    assert "default" in times and any("lattice_method=1" in k for k in times)
    # per-grid tiles are timed exactly when the stencil won
    assert any(k.startswith("grid0=") for k in times) == AT.uses_stencil(summary["shared"])
    t2, s2, times2 = AT.autotune_batch(boxes, pos, q, counts, reps=2, **kw)
    assert t2 == tunings and s2 == summary and "cached" in times2
    mk = lambda ts: [MSM(box=L, periodic=True, precision="mixed", max_atoms=c, tuning=t, **kw)
                     for L, c, t in zip(boxes, counts, ts)]
    E0, _, F0 = MSMBatch(mk([None] * len(counts))).eval(pos, q, counts)
    # the tuned tunings, and every replica on a non-default tile and the pair clusters
    for ts in [tunings, [{"lattice_txn": 2, "lattice_tyn": 8, "pair_targets": 8, "lattice_method": 1}] * len(counts)]:
        E1, _, F1 = MSMBatch(mk(ts)).eval(pos, q, counts)
        torch.cuda.synchronize()
        assert torch.allclose(E0, E1, rtol=1e-6, atol=0)
        assert_atoms(F1.cpu().numpy(), F0.cpu().numpy(), 1e-5)
    # the batch graph (one launch per stage) with those shapes
    E = torch.zeros(len(counts), dtype=torch.float64, device=dev)
    F = torch.zeros((len(q), 3), dtype=torch.float64, device=dev)
    g = MSMBatch(mk([{"lattice_txn": 2, "lattice_tyn": 8, "pair_targets": 8, "lattice_method": 1}] * len(counts))).graph(
        pos, q, counts, E, None, F)
    g.launch()
    torch.cuda.synchronize()
    g.close()
    assert torch.allclose(E0, E, rtol=1e-6, atol=0)
    assert_atoms(F.cpu().numpy(), F0.cpu().numpy(), 1e-5)
