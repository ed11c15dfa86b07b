"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (per comparison, stated here once):
  FP64 path  : energy rel 1e-10, force rel-RMS 1e-9, potential rel-RMS 1e-9.
               Both sides run the same algorithm in double precision; only the
               summation order (and, periodic, two independent Ewald builds of
               the top-level kernel) differ.
  mixed path : energy rel 1e-6, force rel-RMS 1e-5, potential rel-RMS 1e-6
               (the accuracy targets for FP32 pair and grid sums with
               compensated accumulation against the FP64 oracle).
"""
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
    from paper_1402_7216_gb300 import lib
    lib()
    return torch.device("cuda:0")


def plan_for(cfg, precision, n, **kw):
    from paper_1402_7216_gb300 import MSM
    return MSM(box=cfg["box"], periodic=cfg["periodic"], cutoff=cfg["cutoff"], spacing=cfg["spacing"],
               levels=cfg.get("levels", 0), order=cfg["order"], splitting=cfg["split"],
               precision=precision, max_atoms=max(n, 1), **kw)


def oparams(cfg):
    b = cfg["box"]
    return O.Params(box=(b, b, b) if np.isscalar(b) else tuple(b), periodic=cfg["periodic"],
                    cutoff=cfg["cutoff"], spacing=cfg["spacing"], levels=cfg.get("levels", 0),
                    order=cfg["order"], split=cfg["split"])


def gpu_eval(plan, pos, q, dev):
    E, phi, F = plan.eval(torch.tensor(pos, device=dev), torch.tensor(q, device=dev))
    torch.cuda.synchronize()
    plan.check_status()
    return E.item(), phi.cpu().numpy(), F.cpu().numpy()


def assert_close(got, ref, precision, what=""):
    E, phi, F = got
    t = TOL[precision]
    if "E" in ref:
        assert abs(E - ref["E"]) <= t["E"] * abs(ref["E"]), (what, E, ref["E"])
    assert_atoms(F, ref["F"], t["F"], what)
    assert_atoms(phi, ref["phi"], t["phi"], what)


SMALL = [
    dict(name="per-cubic-C2", box=24.0, periodic=True, cutoff=8.0, spacing=1.5, order=3, split=2),
    dict(name="per-quintic-C2", box=24.0, periodic=True, cutoff=8.0, spacing=2.0, order=5, split=2),
    dict(name="per-cubic-C1-l2", box=24.0, periodic=True, cutoff=6.0, spacing=2.0, order=3, split=1, levels=2),
    dict(name="per-quintic-C3-l1", box=24.0, periodic=True, cutoff=6.0, spacing=2.0, order=5, split=3, levels=1),
    dict(name="open-cubic-C2", box=24.0, periodic=False, cutoff=8.0, spacing=2.0, order=3, split=2),
    dict(name="open-quintic-C1", box=24.0, periodic=False, cutoff=7.0, spacing=1.7, order=5, split=1),
    dict(name="open-cubic-C3-l1", box=24.0, periodic=False, cutoff=6.0, spacing=2.0, order=3, split=3, levels=1),
    # 2a/h >= 13, as on the 4.1M-atom box: wide stencils, few grid points per tile
    dict(name="per-quintic-wide", box=30.0, periodic=True, cutoff=10.0, spacing=1.5, order=5, split=2),
    dict(name="open-cubic-wide", box=24.0, periodic=False, cutoff=8.0, spacing=1.2, order=3, split=2),
]


@pytest.mark.parametrize("method", [1, 2], ids=["stencil", "fft"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("cfg", SMALL, ids=[c["name"] for c in SMALL])
def test_small_systems_match_oracle(cfg, precision, method, dev):
    """Both forms of the lattice cutoff (the FFT applies to the periodic cases)."""
    pos, q = make_water_box(cfg["box"], 420, 3, 2, seed=21, periodic=cfg["periodic"])
    ref = O.msm(oparams(cfg), pos, q)
    plan = plan_for(cfg, precision, len(q), tuning={"lattice_method": method})
    # one level has no lattice cutoff at all (only the top level)
    fft = method == 2 and cfg["periodic"] and cfg.get("levels", 0) != 1
    assert plan.lattice_method == ("fft" if fft else "stencil")
    assert plan.levels == ref["geometry"].levels
    assert_close(gpu_eval(plan, pos, q, dev), ref, precision, cfg["name"])


@pytest.mark.parametrize("periodic,method", [(True, 1), (True, 2), (False, 1)],
                         ids=["periodic-stencil", "periodic-fft", "open"])
def test_staged_grids_match_oracle_fp64(periodic, method, dev):
    cfg = dict(box=24.0, periodic=periodic, cutoff=6.0, spacing=1.5, order=5, split=2, levels=3)
    pos, q = make_water_box(24.0, 300, 1, 1, seed=22, periodic=periodic)
    ref = O.msm(oparams(cfg), pos, q, keep_grids=True)
    plan = plan_for(cfg, "fp64", len(q), tuning={"lattice_method": method})
    gpu_eval(plan, pos, q, dev)
    G = ref["geometry"]
    for k in range(G.levels):
        assert plan.dims[k] == G.n[k] and plan.lo[k] == G.lo[k]
        for which, grids in [("q", ref["q_grids"]), ("u", ref["u_grids"])]:
            g = plan.debug_grid(k, which)
            r = grids[k]
            scale = np.abs(r).max()
            assert np.abs(g - r).max() <= 1e-11 * scale, (k, which, np.abs(g - r).max(), scale)


def test_water3k_open_fp64_and_mixed(dev):
    w = WORKLOADS["water3k_open"]
    pos, q = w.make()
    cfg = dict(box=w.box, periodic=False, cutoff=w.cutoff, spacing=w.spacing, order=w.order, split=w.split)
    ref = O.msm(oparams(cfg), pos, q)
    direct = O.direct_sum(pos, q)
    for precision in ["fp64", "mixed"]:
        got = gpu_eval(plan_for(cfg, precision, len(q)), pos, q, dev)
        assert_close(got, ref, precision, precision)
        # and the method's error against the exact Coulomb sum stays in the paper's band
        assert rel_rms(got[2], direct["F"]) < 0.05


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_water23k_periodic(precision, dev):
    w = WORKLOADS["water23k"]
    pos, q = w.make()
    cfg = dict(box=w.box, periodic=True, cutoff=w.cutoff, spacing=w.spacing, order=w.order, split=w.split)
    ref = O.msm(oparams(cfg), pos, q)
    plan = plan_for(cfg, precision, len(q))
    assert plan.dims[0] == (32, 32, 32) and plan.levels == 3
    assert_close(gpu_eval(plan, pos, q, dev), ref, precision)


def test_edge_cases(dev):
    cfg = dict(box=20.0, periodic=True, cutoff=6.0, spacing=2.0, order=3, split=2)
    # no atoms
    plan = plan_for(cfg, "mixed", 16)
    E, _, _ = plan.eval(torch.zeros((0, 3), dtype=torch.float64, device=dev),
                        torch.zeros(0, dtype=torch.float64, device=dev))
    assert E.item() == 0.0
    # one atom, two atoms, atoms exactly on grid points and on the periodic boundary
    for pos in [np.array([[3.3, 4.4, 5.5]]),
                np.array([[2.0, 4.0, 6.0], [18.0, 0.0, 20.0 - 1e-12]]),
                np.array([[0.0, 0.0, 0.0], [2.0, 2.0, 2.0], [10.0, 12.0, 2.0], [19.999999, 8.0, 4.0]])]:
        q = np.resize(np.array([1.0, -0.5, 0.25, -0.75]), len(pos))
        ref = O.msm(oparams(cfg), pos, q)
        for precision in ["fp64", "mixed"]:
            got = gpu_eval(plan_for(cfg, precision, len(q)), pos, q, dev)
            tol = TOL[precision]
            # few atoms: the forces are tiny differences (e.g. a lone atom's grid
            # self force), so they are compared on the scale of a unit-charge
            # interaction at one grid spacing, 1/h^2
            fscale = 1.0 / cfg["spacing"] ** 2
            assert abs(got[0] - ref["E"]) <= tol["E"] * (abs(ref["E"]) + 1.0)
            np.testing.assert_allclose(got[2], ref["F"], rtol=0, atol=tol["F"] * fscale)
    # open box: atoms on the faces x = 0 and x = L
    ocfg = dict(box=20.0, periodic=False, cutoff=6.0, spacing=2.0, order=5, split=2)
    pos = np.array([[0.0, 0.0, 0.0], [20.0, 20.0, 20.0], [20.0, 0.0, 10.0], [4.0, 6.0, 8.0]])
    q = np.array([1.0, -1.0, 0.5, -0.5])
    ref = O.msm(oparams(ocfg), pos, q)
    got = gpu_eval(plan_for(ocfg, "fp64", 4), pos, q, dev)
    assert abs(got[0] - ref["E"]) <= 1e-10 * abs(ref["E"])
    # sparse and dense cells: a cluster far denser than water (many > 32-atom cells) plus empty space
    rng = np.random.default_rng(3)
    pos = np.vstack([rng.uniform(2.0, 6.0, (700, 3)), rng.uniform(0.0, 20.0, (37, 3))])
    q = rng.uniform(-1, 1, len(pos))
    ref = O.msm(oparams(cfg), pos, q)
    for precision in ["fp64", "mixed"]:
        got = gpu_eval(plan_for(cfg, precision, len(q)), pos, q, dev)
        assert abs(got[0] - ref["E"]) <= 10 * TOL[precision]["E"] * abs(ref["E"])
        assert_atoms(got[2], ref["F"], 10 * TOL[precision]["F"])


def test_device_errors_are_reported(dev):
    from paper_1402_7216_gb300 import MSMError
    ocfg = dict(box=20.0, periodic=False, cutoff=6.0, spacing=2.0, order=3, split=2)
    plan = plan_for(ocfg, "mixed", 8)
    pos = torch.tensor([[1.0, 2.0, 3.0], [25.0, 1.0, 1.0]], dtype=torch.float64, device=dev)
    q = torch.tensor([1.0, -1.0], dtype=torch.float64, device=dev)
    plan.eval(pos, q)
    assert plan.status() == -4                         # atom outside the open box
    assert plan.status() == 0                          # cleared after reading
    pos[1, 0] = float("nan")
    plan.eval(pos, q)
    assert plan.status() == -5                         # non-finite input
    with pytest.raises(MSMError) as e:
        plan.eval(torch.zeros((9, 3), dtype=torch.float64, device=dev),
                  torch.zeros(9, dtype=torch.float64, device=dev))
    assert e.value.code == -9                          # more atoms than the plan holds
    fresh = plan_for(ocfg, "mixed", 8)
    with pytest.raises(MSMError):
        fresh.backward(torch.ones((), dtype=torch.float64, device=dev))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_backward_adjoint_matches_forward_outputs(precision, dev):
    from paper_1402_7216_gb300 import MSMEnergy
    cfg = dict(box=24.0, periodic=True, cutoff=8.0, spacing=2.0, order=5, split=2)
    pos, q = make_water_box(24.0, 400, 2, 2, seed=23, periodic=True)
    plan = plan_for(cfg, precision, len(q))
    E, phi, F = plan.eval(torch.tensor(pos, device=dev), torch.tensor(q, device=dev))
    tp = torch.tensor(pos, device=dev, requires_grad=True)
    tq = torch.tensor(q, device=dev, requires_grad=True)
    E2 = MSMEnergy.apply(tp, tq, plan)
    (3.0 * E2).backward()
    t = TOL[precision]
    # repeat of the same forward: the mixed path is bit-reproducible (index
    # order inside cells, fixed-point charge grid, no atomic float sums); the
    # FP64 path still adds anterpolation patches with FP64 atomics
    if precision == "mixed":
        assert E2.item() == E.item()
    else:
        assert abs(E2.item() - E.item()) <= 1e-12 * abs(E.item())
    assert_atoms(tp.grad.cpu().numpy(), -3.0 * F.cpu().numpy(), t["F"])
    assert_atoms(tq.grad.cpu().numpy(), 3.0 * phi.cpu().numpy(), t["phi"])
    ref = O.msm(oparams(cfg), pos, q)
    assert_atoms(-tp.grad.cpu().numpy() / 3.0, ref["F"], t["F"])


def test_backward_finite_differences_water23k_fp64(dev):
    """Central differences (step 1e-4 A) of the FP64 GPU energy on 64 random
    atoms against the adjoint gradient."""
    from paper_1402_7216_gb300 import MSMEnergy
    w = WORKLOADS["water23k"]
    pos, q = w.make()
    cfg = dict(box=w.box, periodic=True, cutoff=w.cutoff, spacing=w.spacing, order=w.order, split=w.split)
    plan = plan_for(cfg, "fp64", len(q))
    tp = torch.tensor(pos, device=dev, requires_grad=True)
    tq = torch.tensor(q, device=dev)
    MSMEnergy.apply(tp, tq, plan).backward()
    grad = tp.grad.cpu().numpy()
    rng = np.random.default_rng(24)
    step = 1e-4
    base = torch.tensor(pos, device=dev)
    for i in rng.choice(len(q), 64, replace=False):
        d = int(rng.integers(3))
        pp, pm = base.clone(), base.clone()
        pp[i, d] += step
        pm[i, d] -= step
        Ep = plan.eval(pp, tq, want_phi=False, want_force=False)[0].item()
        Em = plan.eval(pm, tq, want_phi=False, want_force=False)[0].item()
        fd = (Ep - Em) / (2 * step)
        assert abs(fd - grad[i, d]) <= 1e-6 + 1e-6 * abs(grad[i, d]), (i, d, fd, grad[i, d])


def test_host_entry_point_matches_device(dev):
    cfg = dict(box=24.0, periodic=True, cutoff=8.0, spacing=2.0, order=3, split=2)
    pos, q = make_water_box(24.0, 400, 0, 0, seed=25, periodic=True)
    plan = plan_for(cfg, "mixed", len(q))
    Ed, phid, Fd = gpu_eval(plan, pos, q, dev)
    Eh, phih, Fh = plan.eval_host(torch.tensor(pos).pin_memory(), torch.tensor(q).pin_memory(),
                                  want_phi=True, want_force=True)
    # same inputs, same kernels, and the mixed path sums in an order fixed by
    # the input alone: bit-identical
    assert Eh.item() == Ed
    assert np.array_equal(Fh.numpy(), Fd) and np.array_equal(phih.numpy(), phid)


def test_host_entry_point_reports_device_errors_once(dev):
    """msm_eval_host returns the device status of its own call (an atom
    outside an open box) and clears it: the next good call succeeds."""
    from paper_1402_7216_gb300 import MSMError
    ocfg = dict(box=20.0, periodic=False, cutoff=6.0, spacing=2.0, order=3, split=2)
    plan = plan_for(ocfg, "mixed", 8)
    pos = torch.tensor([[1.0, 2.0, 3.0], [25.0, 1.0, 1.0]], dtype=torch.float64).pin_memory()
    q = torch.tensor([1.0, -1.0], dtype=torch.float64).pin_memory()
    with pytest.raises(MSMError) as e:
        plan.eval_host(pos, q)
    assert e.value.code == -4
    pos[1, 0] = 5.0
    E = plan.eval_host(pos, q)[0]
    assert E.item() < 0.0                                   # two opposite charges 4.6 A apart
    assert plan.status() == 0


def test_repeatable(dev):
    """Two evaluations of the same input: bit-identical on the mixed path
    (binning puts each cell's atoms in input-index order, the charge grid is
    exact fixed point, split lattice levels add their parts in order), also
    on a small box whose coarse levels split their lattice sums and on a
    dense cluster; the FP64 path within 1e-13 (FP64 atomic patch sums)."""
    cfg = dict(box=24.0, periodic=True, cutoff=8.0, spacing=2.0, order=5, split=2)
    pos, q = make_water_box(24.0, 400, 2, 2, seed=26, periodic=True)
    rng = np.random.default_rng(26)
    dense = np.vstack([rng.uniform(2.0, 7.0, (900, 3)), rng.uniform(0.0, 24.0, (100, 3))])
    dq = rng.uniform(-1, 1, len(dense))
    for precision, tol in [("fp64", 1e-13), ("mixed", 0.0)]:
        for P, Q in [(pos, q), (dense, dq)]:
            plan = plan_for(cfg, precision, len(Q))
            a = gpu_eval(plan, P, Q, dev)
            b = gpu_eval(plan, P, Q, dev)
            if tol == 0.0:
                assert a[0] == b[0]
                assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
            else:
                assert abs(a[0] - b[0]) <= tol * abs(a[0])
                assert_atoms(a[2], b[2], tol)
            plan.close()


def test_water1m_mixed_on_subsample(dev):
    """The benchmark workload (1,066,628 atoms, quintic, a = 12, h = 2.5) in the
    benchmark's launch configuration: mixed precision against the oracle on a
    4,096-atom spatial subsample, and its energy against the FP64 GPU path."""
    w = WORKLOADS["water1m"]
    pos, q = w.make()
    cfg = dict(box=w.box, periodic=True, cutoff=w.cutoff, spacing=w.spacing, order=w.order, split=w.split)
    sub = spatial_subsample(pos, (w.box,) * 3, 4096, seed=1)
    ref = O.msm(oparams(cfg), pos, q, targets=sub)
    got = gpu_eval(plan_for(cfg, "mixed", len(q)), pos, q, dev)
    assert_atoms(got[2][sub], ref["F"], TOL["mixed"]["F"])
    assert_atoms(got[1][sub], ref["phi"], TOL["mixed"]["phi"])
    got64 = gpu_eval(plan_for(cfg, "fp64", len(q)), pos, q, dev)
    assert_atoms(got64[2][sub], ref["F"], TOL["fp64"]["F"])
    assert abs(got[0] - got64[0]) <= TOL["mixed"]["E"] * abs(got64[0])


def test_anterpolation_large_and_mixed_charges(dev):
    """The mixed path sums patch charges in fixed point and routes large
    charges (|q| >= 2^10, or |q| * atoms-per-patch > 2^18) straight to the FP64
    grid; both routes, in one system, must match the oracle."""
    cfg = dict(box=24.0, periodic=True, cutoff=8.0, spacing=2.0, order=5, split=2)
    pos, q = make_water_box(24.0, 420, 3, 2, seed=23, periodic=True)
    rng = np.random.default_rng(23)
    scale = rng.choice([1.0, 300.0, 2500.0], size=len(q) // 3 + 1).repeat(3)[: len(q)]
    q = q * scale
    ref = O.msm(oparams(cfg), pos, q)
    for precision in ["fp64", "mixed"]:
        assert_close(gpu_eval(plan_for(cfg, precision, len(q)), pos, q, dev), ref, precision, precision)


def test_overlap_on_and_off_agree(dev):
    """The forward pass with the grid passes on the plan's side stream
    (concurrent with the pair sums) and with every stage in turn on the
    caller's stream: bit-identical on the mixed path (within 1e-13 on the
    FP64 path), and both match the oracle."""
    cfg = dict(box=30.0, periodic=True, cutoff=9.0, spacing=2.0, order=5, split=2)
    pos, q = make_water_box(30.0, 850, 3, 3, seed=27, periodic=True)
    ref = O.msm(oparams(cfg), pos, q)
    for precision, tol in [("fp64", 1e-13), ("mixed", 0.0)]:
        plan = plan_for(cfg, precision, len(q))
        plan.set_overlap(False)
        a = gpu_eval(plan, pos, q, dev)
        plan.set_overlap(True)
        b = gpu_eval(plan, pos, q, dev)
        if tol == 0.0:  # the same sums in the same order on either stream layout
            assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
        else:
            assert abs(a[0] - b[0]) <= tol * abs(a[0])
            assert_atoms(a[2], b[2], tol)
            assert_atoms(a[1], b[1], tol)
        assert_close(b, ref, precision, precision)


def test_stencil_wider_than_the_lattice_window_is_unsupported(dev):
    """2a/h beyond the lattice kernel's shared-memory window is refused at
    plan creation (UNSUPPORTED), not at the first evaluation."""
    from paper_1402_7216_gb300 import MSMError
    # capacity for cells a/2 wide, so that the anterpolation patch fits and
    # the stencil is what decides
    wide = dict(box=40.0, periodic=False, cutoff=12.0, order=3, split=2)
    cap = 10000
    for precision, h in [("mixed", 0.35), ("fp64", 0.85)]:   # 2a/h = 68.6 and 28.2
        with pytest.raises(MSMError) as e:
            plan_for(dict(wide, spacing=h), precision, cap)
        assert e.value.code == -2
    plan = plan_for(dict(wide, spacing=0.85), "mixed", cap)  # fits the FP32 window
    pos = torch.tensor([[10.0, 10.0, 10.0], [13.0, 10.0, 10.0]], dtype=torch.float64, device=dev)
    q = torch.tensor([1.0, -1.0], dtype=torch.float64, device=dev)
    E = plan.eval(pos, q)[0]
    assert abs(E + 1.0 / 3.0) < 1e-3 * (1.0 / 3.0)   # two opposite charges 3 A apart


def test_autograd_two_applies_on_one_plan(dev):
    """Two MSMEnergy.apply calls on one plan before one backward: the second
    forward reuses the plan's buffers, so the first call's backward must
    recompute its own forward (forward ids) and both gradients must be those
    of their own inputs.  The low-level adjoint of a stale forward id is
    refused with STALE_FORWARD."""
    from paper_1402_7216_gb300 import MSMEnergy, MSMError
    cfg = dict(box=24.0, periodic=True, cutoff=8.0, spacing=2.0, order=3, split=2)
    pos1, q1 = make_water_box(24.0, 400, 2, 2, seed=31, periodic=True)
    pos2, q2 = make_water_box(24.0, 380, 1, 1, seed=32, periodic=True)
    for precision in ["fp64", "mixed"]:
        t = TOL[precision]
        plan = plan_for(cfg, precision, max(len(q1), len(q2)))
        _, phi1, F1 = gpu_eval(plan, pos1, q1, dev)
        _, phi2, F2 = gpu_eval(plan, pos2, q2, dev)
        p1 = torch.tensor(pos1, device=dev, requires_grad=True)
        c1 = torch.tensor(q1, device=dev, requires_grad=True)
        p2 = torch.tensor(pos2, device=dev, requires_grad=True)
        c2 = torch.tensor(q2, device=dev, requires_grad=True)
        E1 = MSMEnergy.apply(p1, c1, plan)
        E2 = MSMEnergy.apply(p2, c2, plan)
        (E1 + 2.0 * E2).backward()
        assert_atoms(-p1.grad.cpu().numpy(), F1, t["F"], "first apply")
        assert_atoms(c1.grad.cpu().numpy(), phi1, t["phi"], "first apply")
        assert_atoms(-p2.grad.cpu().numpy(), 2.0 * F2, t["F"], "second apply")
        assert_atoms(c2.grad.cpu().numpy(), 2.0 * phi2, t["phi"], "second apply")
        # the C ABI refuses the adjoint of a forward whose buffers were reused
        plan.eval(torch.tensor(pos1, device=dev), torch.tensor(q1, device=dev))
        fid = plan.forward_id()
        plan.eval(torch.tensor(pos2, device=dev), torch.tensor(q2, device=dev))
        assert plan.forward_id() == fid + 1
        g = torch.ones((), dtype=torch.float64, device=dev)
        with pytest.raises(MSMError) as e:
            plan.backward(g, forward_id=fid)
        assert e.value.code == -11
        gp, _ = plan.backward(g, forward_id=fid + 1)
        torch.cuda.synchronize()
        assert_atoms(-gp.cpu().numpy(), F2, t["F"], "latest forward")
        # the cutoff method leaves no MSM forward to differentiate
        plan.cutoff_eval(torch.tensor(pos2, device=dev), torch.tensor(q2, device=dev))
        assert plan.forward_id() == 0
        plan.close()
