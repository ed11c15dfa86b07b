"""Velocity Verlet MD around the MSM force (msm_md_run, Sec. "Molecular
Dynamics") against the oracle's MD (the same scheme around the FP64 oracle's
MSM force), and the properties the thesis expects of MSM dynamics: energy
conserved (smooth, continuous forces), momentum fluctuating without drift.

Tolerances after 20 steps of a 48-ion system: FP64 plan positions and
velocities 1e-10 absolute, energies 1e-10 relative (same arithmetic, other
summation order); mixed plan positions 1e-5 A, velocity changes rel-RMS 1e-4,
energies 1e-5 relative (FP32 pairs and grids, force rel-RMS ~5e-7 per step).
"""
import numpy as np
import pytest
import torch

from synth import make_ion_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def make_plan(L, n, precision, periodic=True, cutoff=6.0, spacing=2.0, order=3):
    from paper_1402_7216_gb300 import MSM
    return MSM(box=L, periodic=periodic, cutoff=cutoff, spacing=spacing, order=order, splitting=2,
               precision=precision, max_atoms=max(n, 1))


def oparams(L, periodic=True, cutoff=6.0, spacing=2.0, order=3):
    import oracle as O
    return O.Params(box=(L,) * 3, periodic=periodic, cutoff=cutoff, spacing=spacing, order=order, split=2)


def gpu_md(plan, pos, vel, im, q, dt, nsteps, dev):
    tp, tv = torch.tensor(pos, device=dev), torch.tensor(vel, device=dev)
    ti, tq = torch.tensor(im, device=dev), torch.tensor(q, device=dev)
    F, rec = plan.md_run(tp, tv, ti, tq, dt, nsteps)
    torch.cuda.synchronize()
    plan.check_status()
    return tp.cpu().numpy(), tv.cpu().numpy(), F.cpu().numpy(), rec.cpu().numpy()


def min_image(d, L):
    return d - L * np.round(d / L)


@pytest.mark.parametrize("periodic", [True, False])
def test_md_matches_oracle_fp64_and_mixed(periodic, dev):
    from oracle.md import md_run
    L, n, dt, steps = 16.0, 48, 0.05, 20
    pos, q, im, vel = make_ion_system(L, n, seed=21, kind="salt", periodic=periodic)
    r_o, v_o, F_o, rec_o = md_run(oparams(L, periodic), pos, vel, im, q, dt, steps)
    assert np.abs(min_image(r_o - pos, L)).max() > 0.05      # the ions moved
    for precision in ("fp64", "mixed"):
        r, v, F, rec = gpu_md(make_plan(L, n, precision, periodic), pos, vel, im, q, dt, steps, dev)
        dr = np.abs(min_image(r - r_o, L)).max()
        dv = np.sqrt(((v - v_o) ** 2).sum() / ((v_o - vel) ** 2).sum())
        dE = np.abs(rec[:, :3] - rec_o[:, :3]).max() / np.abs(rec_o[:, :3]).max()
        dP = np.abs(rec[:, 3:] - rec_o[:, 3:]).max()
        if precision == "fp64":
            assert dr < 1e-10 and np.abs(v - v_o).max() < 1e-10 and dE < 1e-10 and dP < 1e-10, (dr, dv, dE, dP)
        else:
            assert dr < 1e-5 and dv < 1e-4 and dE < 1e-5 and dP < 1e-5, (dr, dv, dE, dP)
        if periodic:
            assert r.min() >= 0.0 and r.max() < L                 # wrapped into the box


def test_md_time_reversible_fp64(dev):
    L, n, dt = 20.0, 200, 0.05
    pos, q, im, vel = make_ion_system(L, n, seed=22, kind="plasma")
    plan = make_plan(L, n, "fp64")
    tp, tv = torch.tensor(pos, device=dev), torch.tensor(vel, device=dev)
    ti, tq = torch.tensor(im, device=dev), torch.tensor(q, device=dev)
    F, _ = plan.md_run(tp, tv, ti, tq, dt, 30)
    tv.neg_()
    plan.md_run(tp, tv, ti, tq, dt, 30, force=F)
    torch.cuda.synchronize()
    assert np.abs(min_image(tp.cpu().numpy() - pos, L)).max() < 1e-8
    assert np.abs(-tv.cpu().numpy() - vel).max() < 1e-8


def test_md_energy_conserved_momentum_bounded_mixed(dev):
    """A one-component plasma of 2,000 ions, 400 steps on the mixed plan:
    total energy within 1e-3 of the mean kinetic energy, and the total
    momentum (not conserved by MSM) stays near zero."""
    L, n, dt, steps = 34.0, 2000, 0.05, 400
    pos, q, im, vel = make_ion_system(L, n, seed=23, kind="plasma", dmin=2.5)
    plan = make_plan(L, n, "mixed", cutoff=8.0)
    _, v, _, rec = gpu_md(plan, pos, vel, im, q, dt, steps, dev)
    K = rec[:, 1].mean()
    drift = np.abs(rec[:, 2] - rec[0, 2]).max() / K
    assert drift < 1e-3, drift
    assert np.abs(rec[:, 1] - rec[0, 1]).max() / K > 1e-3     # energy did move between U and K
    p_scale = np.abs(v / im[:, None]).sum()
    assert np.abs(rec[:, 3:]).max() / p_scale < 1e-3


def test_md_graph_capture_and_chunks_match_one_call(dev):
    """Two captured 5-step graphs replayed, and two direct 5-step calls, give
    the trajectory of one 10-step call."""
    L, n, dt = 16.0, 60, 0.05
    pos, q, im, vel = make_ion_system(L, n, seed=24, kind="plasma")
    plan = make_plan(L, n, "fp64")
    ref = gpu_md(plan, pos, vel, im, q, dt, 10, dev)
    tp, tv = torch.tensor(pos, device=dev), torch.tensor(vel, device=dev)
    ti, tq = torch.tensor(im, device=dev), torch.tensor(q, device=dev)
    _, _, F = plan.eval(tp, tq, want_phi=False)
    plan.md_run(tp, tv, ti, tq, dt, 5, force=F)
    plan.md_run(tp, tv, ti, tq, dt, 5, force=F)
    torch.cuda.synchronize()
    np.testing.assert_allclose(tp.cpu().numpy(), ref[0], atol=1e-11)
    # graph: capture 5 steps on static buffers, replay twice
    gp, gv = torch.tensor(pos, device=dev), torch.tensor(vel, device=dev)
    _, _, gF = plan.eval(gp, tq, want_phi=False)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        _, grec = plan.md_run(gp, gv, ti, tq, dt, 5, force=gF)
    # capture only records: the buffers still hold the start state
    np.testing.assert_array_equal(gp.cpu().numpy(), pos)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    plan.check_status()
    np.testing.assert_allclose(gp.cpu().numpy(), ref[0], atol=1e-11)
    np.testing.assert_allclose(gv.cpu().numpy(), ref[1], atol=1e-11)
    np.testing.assert_allclose(grec.cpu().numpy(), ref[3][5:], rtol=1e-11, atol=1e-12)


def test_md_fixed_atoms_zero_steps_and_errors(dev):
    from paper_1402_7216_gb300 import MSMError
    L, n = 16.0, 40
    pos, q, im, vel = make_ion_system(L, n, seed=25, kind="plasma")
    im[:5] = 0.0
    vel[:5] = 0.0
    plan = make_plan(L, n, "mixed")
    r, v, _, rec = gpu_md(plan, pos, vel, im, q, 0.05, 10, dev)
    np.testing.assert_array_equal(r[:5], pos[:5])            # fixed: no kick, no drift
    np.testing.assert_array_equal(v[:5], 0.0)
    assert np.abs(r[5:] - pos[5:]).max() > 1e-3
    tp, tv = torch.tensor(pos, device=dev), torch.tensor(vel, device=dev)
    ti, tq = torch.tensor(im, device=dev), torch.tensor(q, device=dev)
    F, rec0 = plan.md_run(tp, tv, ti, tq, 0.05, 0)
    torch.cuda.synchronize()
    assert rec0.shape == (0, 6)
    np.testing.assert_array_equal(tp.cpu().numpy(), pos)
    for dt, steps, code in ((0.05, -1, -1), (float("nan"), 3, -1), (float("inf"), 3, -1)):
        with pytest.raises(MSMError) as e:
            plan.md_run(tp, tv, ti, tq, dt, steps, force=F)
        assert e.value.code == code
    big = make_plan(L, 8, "mixed")                            # capacity 8 < 40 atoms
    with pytest.raises(MSMError) as e:
        big.md_run(tp, tv, ti, tq, 0.05, 1, force=F)
    assert e.value.code == -9


def test_md_atom_leaving_an_open_box_is_reported(dev):
    """An open box has no wrap: an atom driven out of [0, L] is reported by
    the next evaluation's device check through msm_status (no fault)."""
    from paper_1402_7216_gb300 import MSMError
    L, n = 16.0, 40
    pos, q, im, vel = make_ion_system(L, n, seed=26, kind="plasma", periodic=False)
    vel[0] = (40.0, 0.0, 0.0)                             # 2 A per step along +x
    plan = make_plan(L, n, "mixed", periodic=False)
    tp, tv, ti, tq = (torch.tensor(a, device=dev) for a in (pos, vel, im, q))
    plan.md_run(tp, tv, ti, tq, 0.05, 10)
    torch.cuda.synchronize()
    with pytest.raises(MSMError) as e:
        plan.check_status()
    assert e.value.code == -4
    assert plan.status() == 0                             # cleared once read


def test_md_with_no_atoms(dev):
    """n = 0: every step's record is zero and nothing is touched."""
    plan = make_plan(16.0, 4, "mixed")
    z3 = torch.zeros((0, 3), dtype=torch.float64, device=dev)
    z1 = torch.zeros(0, dtype=torch.float64, device=dev)
    F, rec = plan.md_run(z3, z3.clone(), z1, z1.clone(), 0.05, 3, force=z3.clone())
    torch.cuda.synchronize()
    plan.check_status()
    assert rec.shape == (3, 6)
    assert torch.all(rec == 0.0)
