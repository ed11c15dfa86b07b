"""The cutoff method (the parareal section's coarse propagator G: the Coulomb
law within a constant cutoff) through msm_cutoff_eval, against the FP64
oracle's brute-force cutoff sum.  The cutoff is hard, so a pair within
rounding of r = a is inside on one side and outside on the other: such atoms
are left out of the element-wise comparison (both answers are valid) and the
energy tolerance grows by the largest change a flipped pair can make.

Tolerances: FP64 plan energy rel 1e-10, force/potential rel-RMS 1e-9 (same
sum, other order); mixed plan energy rel 1e-6, force rel-RMS 1e-5, potential
rel-RMS 1e-6 (FP32 pair sums with compensated accumulation)."""
import numpy as np
import pytest
import torch

import oracle as O
from conftest import assert_atoms, rel_rms
from synth import make_water_box, spatial_subsample, WORKLOADS

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(E=1e-10, F=1e-9, phi=1e-9), "mixed": dict(E=1e-6, F=1e-5, phi=1e-6)}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def plan(box, periodic, cutoff, precision, n):
    from paper_1402_7216_gb300 import MSM
    return MSM(box=box, periodic=periodic, cutoff=cutoff, spacing=2.0, order=3, splitting=2,
               precision=precision, max_atoms=max(n, 1))


def run(p, pos, q, dev):
    E, phi, F = p.cutoff_eval(torch.tensor(pos, device=dev), torch.tensor(q, device=dev))
    torch.cuda.synchronize()
    p.check_status()
    return E.item(), phi.cpu().numpy(), F.cpu().numpy()


def edge_pairs(pos, q, box, periodic, a, targets=None, delta=1e-5):
    """Pairs whose distance lies within delta of the cutoff.  Whether such a
    pair is inside is decided by rounding (FP32 on the mixed plan, FP64 in
    the oracle), so both answers are valid: returns the set of target
    indices (positions in `targets`, or atoms) that have one, and the
    largest energy change a flipped decision can make, sum |q_i q_j| / a."""
    from scipy.spatial import cKDTree
    L = np.full(3, box)
    tree = cKDTree(np.mod(pos, L) if periodic else pos, boxsize=L if periodic else None)
    tgt = np.arange(len(q)) if targets is None else np.asarray(targets)
    hits, dE = set(), 0.0
    for t, i in enumerate(tgt):
        for j in tree.query_ball_point(np.mod(pos[i], L) if periodic else pos[i], a + delta):
            if j == i:
                continue
            d = pos[i] - pos[j]
            if periodic:
                d -= L * np.round(d / L)
            if abs(np.sqrt(d @ d) - a) < delta:
                hits.add(t)
                dE += abs(q[i] * q[j]) / a / 2.0
    return hits, dE


def check(got, ref, precision, pos, q, box, periodic, a):
    t = TOL[precision]
    hits, dE = edge_pairs(pos, q, box, periodic, a) if precision == "mixed" else (set(), 0.0)
    assert abs(got[0] - ref["E"]) <= t["E"] * abs(ref["E"]) + dE, (got[0], ref["E"])
    keep = np.array([i for i in range(len(q)) if i not in hits], dtype=int)
    assert len(keep) >= 0.99 * len(q)
    assert_atoms(got[2][keep], ref["F"][keep], t["F"])
    assert_atoms(got[1][keep], ref["phi"][keep], t["phi"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("periodic,box,cutoff", [(True, 24.0, 8.0), (True, 30.0, 12.0), (False, 24.0, 7.0)])
def test_cutoff_matches_oracle(periodic, box, cutoff, precision, dev):
    pos, q = make_water_box(box, 430, 3, 3, seed=81, periodic=periodic)
    P = O.Params(box=(box,) * 3, periodic=periodic, cutoff=cutoff, spacing=2.0)
    check(run(plan(box, periodic, cutoff, precision, len(q)), pos, q, dev), O.cutoff_sum(P, pos, q), precision,
          pos, q, box, periodic, cutoff)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cutoff_water23k(precision, dev):
    w = WORKLOADS["water23k"]
    pos, q = w.make()
    P = O.Params(box=(w.box,) * 3, periodic=True, cutoff=w.cutoff, spacing=w.spacing)
    check(run(plan(w.box, True, w.cutoff, precision, len(q)), pos, q, dev), O.cutoff_sum(P, pos, q), precision,
          pos, q, w.box, True, w.cutoff)


def test_cutoff_water1m_subsample(dev):
    """The benchmark system (1,066,628 atoms, a = 12): mixed precision against
    the oracle on a 4,096-atom spatial subsample."""
    w = WORKLOADS["water1m"]
    pos, q = w.make()
    sub = spatial_subsample(pos, (w.box,) * 3, 4096, seed=2)
    P = O.Params(box=(w.box,) * 3, periodic=True, cutoff=w.cutoff, spacing=w.spacing)
    ref = O.cutoff_sum(P, pos, q, targets=sub)
    E, phi, F = run(plan(w.box, True, w.cutoff, "mixed", len(q)), pos, q, dev)
    hits, _ = edge_pairs(pos, q, w.box, True, w.cutoff, targets=sub)
    keep = np.array([t for t in range(len(sub)) if t not in hits], dtype=int)
    assert len(keep) >= 0.98 * len(sub)   # ~4 pi a^2 (2 delta) rho = 0.4 % of the atoms expected
    assert_atoms(F[sub][keep], ref["F"][keep], TOL["mixed"]["F"])
    assert_atoms(phi[sub][keep], ref["phi"][keep], TOL["mixed"]["phi"])


def test_cutoff_edge_cases(dev):
    from paper_1402_7216_gb300 import MSMError
    p = plan(20.0, True, 6.0, "mixed", 8)
    E, _, _ = p.cutoff_eval(torch.zeros((0, 3), dtype=torch.float64, device=dev),
                            torch.zeros(0, dtype=torch.float64, device=dev))
    assert E.item() == 0.0
    # two charges inside and beyond the cutoff (minimum image across the boundary)
    for x2, inside in [(4.0, True), (16.5, True), (10.0, False)]:   # r = 3, 4.5 (image), 9
        pos = np.array([[1.0, 5.0, 5.0], [x2, 5.0, 5.0]])
        q = np.array([0.6, -0.9])
        E, phi, F = run(plan(20.0, True, 6.0, "fp64", 2), pos, q, dev)
        d = 1.0 - x2
        d -= 20.0 * np.round(d / 20.0)
        r = abs(d)
        assert E == pytest.approx(0.6 * -0.9 / r if inside else 0.0, rel=1e-12, abs=1e-15)
    # the adjoint of an MSM evaluation is not available after a cutoff evaluation
    with pytest.raises(MSMError):
        p.backward(torch.ones((), dtype=torch.float64, device=dev))
