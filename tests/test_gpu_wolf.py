"""Wolf summation (damped, shifted force; the parareal section's other coarse
function G) through msm_wolf_eval, against the FP64 oracle's brute-force
Wolf sum.  The pair potential and its derivative vanish at the cutoff, so a
pair within rounding of r = R changes nothing measurable and every atom is
compared.

Tolerances: FP64 plan energy rel 1e-10, force/potential rel-RMS 1e-9 (same
sum, other order); mixed plan energy rel 1e-6, force rel-RMS 1e-5, potential
rel-RMS 1e-6 (FP32 pair sums with compensated accumulation; erfc by
Abramowitz and Stegun 7.1.26, |error| < 1.5e-7, which moves the potential by
~2e-7 rel-RMS on water), each with the per-atom bound of
conftest.assert_atoms."""
import numpy as np
import pytest
import torch

import oracle as O
from conftest import assert_atoms
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


def run(p, pos, q, alpha, dev):
    E, phi, F = p.wolf_eval(torch.tensor(pos, device=dev), torch.tensor(q, device=dev), alpha)
    torch.cuda.synchronize()
    p.check_status()
    return E.item(), phi.cpu().numpy(), F.cpu().numpy()


def check(got, ref, precision, what=""):
    t = TOL[precision]
    assert abs(got[0] - ref["E"]) <= t["E"] * abs(ref["E"]), (what, got[0], ref["E"])
    assert_atoms(got[2], ref["F"], t["F"], what)
    assert_atoms(got[1], ref["phi"], t["phi"], what)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("periodic,box,cutoff,alpha", [(True, 24.0, 8.0, 0.25), (True, 30.0, 12.0, 0.2),
                                                        (False, 24.0, 7.0, 0.3), (True, 24.0, 9.0, 0.0)])
def test_wolf_matches_oracle(periodic, box, cutoff, alpha, precision, dev):
    pos, q = make_water_box(box, 430, 3, 3, seed=91, periodic=periodic)
    P = O.Params(box=(box,) * 3, periodic=periodic, cutoff=cutoff, spacing=2.0)
    check(run(plan(box, periodic, cutoff, precision, len(q)), pos, q, alpha, dev), O.wolf_sum(P, pos, q, alpha),
          precision, (periodic, box, cutoff, alpha))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_wolf_water23k(precision, dev):
    w = WORKLOADS["water23k"]
    pos, q = w.make()
    P = O.Params(box=(w.box,) * 3, periodic=True, cutoff=w.cutoff, spacing=w.spacing)
    check(run(plan(w.box, True, w.cutoff, precision, len(q)), pos, q, 0.24, dev), O.wolf_sum(P, pos, q, 0.24),
          precision)


def test_wolf_water1m_subsample(dev):
    """The benchmark system (1,066,628 atoms, R = 12, alpha = 0.2): mixed
    precision against the oracle on a 4,096-atom spatial subsample."""
    w = WORKLOADS["water1m"]
    pos, q = w.make()
    sub = spatial_subsample(pos, (w.box,) * 3, 4096, seed=3)
    P = O.Params(box=(w.box,) * 3, periodic=True, cutoff=w.cutoff, spacing=w.spacing)
    ref = O.wolf_sum(P, pos, q, 0.2, targets=sub)
    E, phi, F = run(plan(w.box, True, w.cutoff, "mixed", len(q)), pos, q, 0.2, dev)
    assert_atoms(F[sub], ref["F"], TOL["mixed"]["F"])
    assert_atoms(phi[sub], ref["phi"], TOL["mixed"]["phi"])


def test_wolf_md_matches_oracle_trajectory(dev):
    """Velocity Verlet with the Wolf force (method "wolf", the plan's alpha):
    20 steps of a small plasma on the FP64 plan follow the oracle's
    integrator around the oracle's Wolf sum."""
    from oracle.md import velocity_verlet
    from synth import make_ion_system
    L, n = 20.0, 400
    pos, q, im, vel = make_ion_system(L, n, seed=93, kind="plasma", dmin=1.5)
    p = plan(L, True, 7.0, "fp64", n)
    p.set_wolf_alpha(0.3)
    P = O.Params(box=(L,) * 3, periodic=True, cutoff=7.0, spacing=2.0)

    def force(r):
        out = O.wolf_sum(P, r, q, 0.3)
        return out["F"], out["E"]
    r_ref, v_ref, _, _ = velocity_verlet(force, pos, vel, im, 0.02, 20, wrap=lambda r: r - L * np.floor(r / L))
    tp, tv, ti, tq = (torch.tensor(a, device=dev) for a in (pos, vel, im, q))
    _, _, F0 = p.wolf_eval(tp, tq, 0.3)
    p.md_run(tp, tv, ti, tq, 0.02, 20, force=F0, method="wolf")
    torch.cuda.synchronize()
    p.check_status()
    d = tp.cpu().numpy() - r_ref
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 1e-10
    assert np.abs(tv.cpu().numpy() - v_ref).max() < 1e-10


def test_wolf_edge_cases_and_arguments(dev):
    from paper_1402_7216_gb300 import MSMError
    p = plan(20.0, True, 6.0, "mixed", 8)
    E, _, _ = p.wolf_eval(torch.zeros((0, 3), dtype=torch.float64, device=dev),
                          torch.zeros(0, dtype=torch.float64, device=dev), 0.3)
    assert E.item() == 0.0
    # two charges inside and beyond the cutoff: the pair term, plus the self terms
    alpha, R = 0.3, 6.0
    cs = O.wolf_self_coefficient(alpha, R)
    for x2 in [4.0, 16.5, 10.0]:   # r = 3, 4.5 (minimum image), 9 (beyond R)
        pos = np.array([[1.0, 5.0, 5.0], [x2, 5.0, 5.0]])
        q = np.array([0.6, -0.9])
        E, phi, F = run(plan(20.0, True, R, "fp64", 2), pos, q, alpha, dev)
        d = 1.0 - x2
        d -= 20.0 * np.round(d / 20.0)
        v, _ = O.wolf_pair(alpha, R, abs(d))
        assert E == pytest.approx(0.6 * -0.9 * v - cs * (0.36 + 0.81), rel=1e-12)
    for bad in [-0.1, float("nan"), float("inf")]:
        with pytest.raises(MSMError) as e:
            p.wolf_eval(torch.zeros((1, 3), dtype=torch.float64, device=dev),
                        torch.zeros(1, dtype=torch.float64, device=dev), bad)
        assert e.value.code == -1
        with pytest.raises(MSMError):
            p.set_wolf_alpha(bad)
    # the adjoint of an MSM evaluation is not available after a Wolf evaluation
    with pytest.raises(MSMError):
        p.backward(torch.ones((), dtype=torch.float64, device=dev))
