"""The largest workload (4.1M atoms, 340 A periodic water box with 0.15 M
NaCl, a = 10, h = 1.5 -> 240^3 finest grid, quintic, 5 levels) at full size:
properties that hold at any size, and the mixed path against the FP64 path
(which the smaller systems pin to the oracle).  Oracle subsample checks at
this size would need the FP64 lattice sum on 13.8M points (~1.6e11 taps) on
the host, so they run on the 1.07M-atom system instead."""
import numpy as np
import pytest
import torch

from conftest import rel_rms
from synth import WORKLOADS

pytestmark = pytest.mark.gpu


def test_water4m_mixed_vs_fp64_and_invariants():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_7216_gb300 import MSM
    dev = torch.device("cuda:0")
    w = WORKLOADS["water4m"]
    pos_h, q_h = w.make()
    assert len(q_h) == 4_100_000 and abs(q_h.sum()) < 1e-9
    pos, q = torch.tensor(pos_h, device=dev), torch.tensor(q_h, device=dev)
    out = {}
    for precision in ["mixed", "fp64"]:
        plan = MSM(box=w.box, periodic=True, cutoff=w.cutoff, spacing=w.spacing, levels=w.levels, order=w.order,
                   splitting=w.split, precision=precision, max_atoms=len(q_h))
        assert plan.dims[0] == (240, 240, 240) and plan.levels == 5
        E, phi, F = plan.eval(pos, q)
        torch.cuda.synchronize()
        plan.check_status()
        out[precision] = (E.item(), phi.cpu().numpy(), F.cpu().numpy())
        plan.close()
    Em, phim, Fm = out["mixed"]
    Ed, phid, Fd = out["fp64"]
    assert abs(Em - Ed) <= 1e-6 * abs(Ed)
    assert rel_rms(Fm, Fd) <= 1e-5
    assert rel_rms(phim, phid) <= 1e-6
    # E = 1/2 sum q phi (the energy reduction against the per-atom outputs)
    assert abs(0.5 * float(np.dot(q_h, phid)) - Ed) <= 1e-10 * abs(Ed)
    # net force small against the force scale (MSM does not conserve momentum exactly)
    assert np.linalg.norm(Fd.sum(0)) < 1e-3 * np.sqrt((Fd ** 2).sum())
