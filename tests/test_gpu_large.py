"""The largest workload (4.1M atoms, 340 A periodic water box with 0.15 M
NaCl, a = 10, h = 1.5 -> 240^3 finest grid, quintic, 5 levels) at full size,
forward and adjoint, with the stencil and with the FFT lattice (240 = 15 x
16: radices 4, 4, 3, 5): properties that hold at any size, and the mixed path
against the FP64 path (which the smaller systems pin to the oracle).  Oracle
checks at this size would need the FP64 lattice sum on 13.8M points (~1.6e11
taps) on the host, so they run on the 1.07M-atom system instead.

The adjoint rebuilds the level-0 potential from the anterpolated adjoint
charges (the forward's level-0 charges scaled) instead of storing any forward
potential; its gradients must equal the
forward's -F and phi (dE/dr = -F, dE/dq = phi) and agree between precisions.
Tolerances: mixed vs FP64 energy 1e-6, force and dE/dr rel-RMS 1e-5,
potential and dE/dq rel-RMS 1e-6, each with the per-atom bound of
conftest.assert_atoms."""
import numpy as np
import pytest
import torch

from conftest import assert_atoms
from synth import WORKLOADS

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method", [1, 2], ids=["stencil", "fft"])
def test_water4m_forward_adjoint_mixed_vs_fp64_and_invariants(method):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_7216_gb300 import MSM
    dev = torch.device("cuda:0")
    w = WORKLOADS["water4m"]
    pos_h, q_h = w.make()
    assert len(q_h) == 4_100_000 and abs(q_h.sum()) < 1e-9
    pos, q = torch.tensor(pos_h, device=dev), torch.tensor(q_h, device=dev)
    gE = torch.full((), 2.0, dtype=torch.float64, device=dev)
    out = {}
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    held = {}
    for precision in ["mixed", "fp64"]:
        plan = MSM(box=w.box, periodic=True, cutoff=w.cutoff, spacing=w.spacing, levels=w.levels, order=w.order,
                   splitting=w.split, precision=precision, max_atoms=len(q_h), tuning={"lattice_method": method})
        assert plan.dims[0] == (240, 240, 240) and plan.levels == 5
        assert plan.lattice_method == {1: "stencil", 2: "fft"}[method]
        E, phi, F = plan.eval(pos, q)
        gp, gq = plan.backward(gE)
        torch.cuda.synchronize()
        plan.check_status()
        held[precision] = free0 - torch.cuda.mem_get_info(dev)[0]
        out[precision] = tuple(t.cpu().numpy() for t in (E, phi, F, gp, gq))
        plan.close()
        del E, phi, F, gp, gq
    Em, phim, Fm, gpm, gqm = out["mixed"]
    Ed, phid, Fd, gpd, gqd = out["fp64"]
    Em, Ed = float(Em), float(Ed)
    # forward: mixed against FP64
    assert abs(Em - Ed) <= 1e-6 * abs(Ed)
    assert_atoms(Fm, Fd, 1e-5, "F")
    assert_atoms(phim, phid, 1e-6, "phi")
    # adjoint: dL/dr = -g F and dL/dq = g phi of the same forward, per precision
    assert_atoms(gpd, -2.0 * Fd, 1e-9, "fp64 dE/dr vs -F")
    assert_atoms(gqd, 2.0 * phid, 1e-9, "fp64 dE/dq vs phi")
    assert_atoms(gpm, -2.0 * Fm, 1e-5, "mixed dE/dr vs -F")
    assert_atoms(gqm, 2.0 * phim, 1e-6, "mixed dE/dq vs phi")
    # ... and across precisions
    assert_atoms(gpm, gpd, 1e-5, "dE/dr mixed vs fp64")
    assert_atoms(gqm, gqd, 1e-6, "dE/dq mixed vs fp64")
    # E = 1/2 sum q phi (the energy reduction against the per-atom outputs)
    assert abs(0.5 * float(np.dot(q_h, phid)) - Ed) <= 1e-10 * abs(Ed)
    # net force small against the force scale (MSM does not conserve momentum exactly)
    assert np.linalg.norm(Fd.sum(0)) < 1e-3 * np.sqrt((Fd ** 2).sum())
    # the plans' device memory (workspace plus the caller's outputs) is far
    # inside the 180 GB budget of this configuration
    assert max(held.values()) < 20e9, held
