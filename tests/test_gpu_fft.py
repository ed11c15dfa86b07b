"""The FFT form of the lattice cutoff (msm_tuning.lattice_method = 2).

On a periodic level the lattice cutoff of Sec. "Multilevel Summation Method"
(u^k = sum over grid points within 2^(k+1) a of g^k q^k) is a cyclic
convolution of the level's charges with the folded stencil, so the CUDA FFT
path must give the oracle's grids and per-atom results within the same
tolerances as the stencil path (FP64: grids 1e-11 of their largest value;
mixed: the stencil path's FP32 tolerances), and agree with the stencil path
of the same plan.  Grid sizes cover radices 2, 4 (16, 32, 96, 256), 3 (24,
12, 6), 7 (14, 7), two odd stages (30 = 2 x 3 x 5, 18 = 2 x 3 x 3) and a
rectangular box.
"""
import numpy as np
import pytest
import torch

import oracle as O
from conftest import assert_atoms
from synth import make_water_box, spatial_subsample, WORKLOADS
from test_gpu_parity import TOL, assert_close, dev, gpu_eval, oparams, plan_for  # noqa: F401

pytestmark = pytest.mark.gpu

FFT = {"lattice_method": 2}
STENCIL = {"lattice_method": 1}

PERIODIC = [
    dict(name="cubic-16", box=24.0, periodic=True, cutoff=8.0, spacing=1.5, order=3, split=2),
    dict(name="quintic-14-radix7", box=21.0, periodic=True, cutoff=6.0, spacing=1.5, order=5, split=2),
    dict(name="quintic-24-radix3-l3", box=36.0, periodic=True, cutoff=9.0, spacing=1.5, order=5, split=2),
    dict(name="cubic-C1-l2", box=24.0, periodic=True, cutoff=6.0, spacing=2.0, order=3, split=1, levels=2),
    dict(name="quintic-C3-l3", box=24.0, periodic=True, cutoff=6.0, spacing=1.5, order=5, split=3, levels=3),
    dict(name="rect-16x14x24", box=(24.0, 21.0, 36.0), periodic=True, cutoff=7.0, spacing=1.5, order=5,
         split=2),
    # explicit level counts leave odd factors 15 = 3 x 5 and 9 = 3 x 3 in the grid sizes
    dict(name="quintic-30-radix15-l2", box=45.0, periodic=True, cutoff=9.0, spacing=1.5, order=5, split=2, levels=2),
    dict(name="cubic-18-radix9-l2", box=27.0, periodic=True, cutoff=7.0, spacing=1.5, order=3, split=2, levels=2),
]


def rect_plan(cfg, precision, n, tuning):
    from paper_1402_7216_gb300 import MSM
    return MSM(box=cfg["box"], periodic=cfg["periodic"], cutoff=cfg["cutoff"], spacing=cfg["spacing"],
               levels=cfg.get("levels", 0), order=cfg["order"], splitting=cfg["split"],
               precision=precision, max_atoms=max(n, 1), tuning=tuning)


def water(cfg, seed, density=0.025):
    """Waters at `density` per cubic length unit (liquid water: 0.033), plus
    three Na+ and two Cl-."""
    nw = int(density * float(np.prod(np.broadcast_to(cfg["box"], (3,)))))
    return make_water_box(cfg["box"], nw, 3, 2, seed=seed, periodic=True)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("cfg", PERIODIC, ids=[c["name"] for c in PERIODIC])
def test_fft_lattice_matches_oracle(cfg, precision, dev):
    pos, q = water(cfg, 41)
    ref = O.msm(oparams(cfg), pos, q)
    plan = rect_plan(cfg, precision, len(q), FFT)
    assert plan.lattice_method == "fft"
    assert plan.levels == ref["geometry"].levels
    assert_close(gpu_eval(plan, pos, q, dev), ref, precision, cfg["name"])


@pytest.mark.parametrize("cfg", PERIODIC[1:3], ids=[c["name"] for c in PERIODIC[1:3]])
def test_fft_staged_grids_match_oracle_fp64(cfg, dev):
    """Every level's u grid (lattice cutoff + prolongation from above) of the
    FP64 FFT path against the oracle's grids."""
    pos, q = water(cfg, 42, 0.02)
    ref = O.msm(oparams(cfg), pos, q, keep_grids=True)
    plan = rect_plan(cfg, "fp64", len(q), FFT)
    assert plan.lattice_method == "fft"
    gpu_eval(plan, pos, q, dev)
    for k in range(ref["geometry"].levels):
        g = plan.debug_grid(k, "u")
        r = ref["u_grids"][k]
        scale = np.abs(r).max()
        assert np.abs(g - r).max() <= 1e-11 * scale, (k, np.abs(g - r).max(), scale)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fft_and_stencil_agree_water23k(precision, dev):
    """Same plan parameters, the two lattice forms: per-atom results within
    the path's tolerance of each other and of the oracle; the adjoint too."""
    w = WORKLOADS["water23k"]
    pos, q = w.make()
    cfg = dict(box=w.box, periodic=True, cutoff=w.cutoff, spacing=w.spacing, order=w.order, split=w.split)
    ref = O.msm(oparams(cfg), pos, q)
    a = plan_for(cfg, precision, len(q), tuning=FFT)
    b = plan_for(cfg, precision, len(q), tuning=STENCIL)
    assert (a.lattice_method, b.lattice_method) == ("fft", "stencil")
    ga, gb = gpu_eval(a, pos, q, dev), gpu_eval(b, pos, q, dev)
    assert_close(ga, ref, precision, "fft")
    t = TOL[precision]
    assert abs(ga[0] - gb[0]) <= t["E"] * abs(gb[0])
    assert_atoms(ga[2], gb[2], t["F"], "F fft vs stencil")
    assert_atoms(ga[1], gb[1], t["phi"], "phi fft vs stencil")
    # the adjoint: dE/dq = phi and dE/dpos = -F hold for both forms
    dt = torch.float64
    P = torch.tensor(pos, device=dev, dtype=dt)
    Q = torch.tensor(q, device=dev, dtype=dt)
    grads = []
    for plan in (a, b):
        plan.eval(P, Q)
        gp, gq = plan.backward(torch.ones((), device=dev, dtype=torch.float64))
        torch.cuda.synchronize()
        plan.check_status()
        grads.append((gp.cpu().numpy(), gq.cpu().numpy()))
    assert_atoms(grads[0][0], -ga[2], t["F"], "grad pos fft")
    assert_atoms(grads[0][1], ga[1], t["phi"], "grad q fft")
    assert_atoms(grads[0][0], grads[1][0], t["F"], "grad pos fft vs stencil")


def test_fft_lattice_is_repeatable(dev):
    """No atomics in the five passes: repeated evaluations are bit-identical."""
    cfg = PERIODIC[2]
    pos, q = water(cfg, 43)
    plan = rect_plan(cfg, "mixed", len(q), FFT)
    first = gpu_eval(plan, pos, q, dev)
    for _ in range(3):
        again = gpu_eval(plan, pos, q, dev)
        assert again[0] == first[0]
        assert np.array_equal(again[1], first[1]) and np.array_equal(again[2], first[2])


def test_fft_request_on_open_plan_keeps_stencil(dev):
    cfg = dict(box=24.0, periodic=False, cutoff=8.0, spacing=2.0, order=3, split=2)
    pos, q = make_water_box(24.0, 300, 1, 1, seed=44, periodic=False)
    plan = plan_for(cfg, "mixed", len(q), tuning=FFT)
    assert plan.lattice_method == "stencil"
    assert_close(gpu_eval(plan, pos, q, dev), O.msm(oparams(cfg), pos, q), "mixed")


def test_fft_water1m_mixed_on_subsample(dev):
    """The 1,066,628-atom benchmark box (levels 96^3 .. 12^3 through the FFT)
    against the oracle on a 4,096-atom spatial subsample."""
    w = WORKLOADS["water1m"]
    pos, q = w.make()
    cfg = dict(box=w.box, periodic=True, cutoff=w.cutoff, spacing=w.spacing, order=w.order, split=w.split)
    sub = spatial_subsample(pos, (w.box,) * 3, 4096, seed=1)
    ref = O.msm(oparams(cfg), pos, q, targets=sub)
    plan = plan_for(cfg, "mixed", len(q), tuning=FFT)
    assert plan.lattice_method == "fft"
    got = gpu_eval(plan, pos, q, dev)
    assert_atoms(got[2][sub], ref["F"], TOL["mixed"]["F"])
    assert_atoms(got[1][sub], ref["phi"], TOL["mixed"]["phi"])


def test_fft_batch_graph_matches_single_plans(dev):
    """Replicas whose plans all took the FFT form: the batched graph runs the
    lattice cutoff of every level of every replica as five launches, and its
    forward and adjoint match each replica's own evaluation (FFT and stencil)
    and the oracle."""
    from paper_1402_7216_gb300 import MSM, MSMBatch
    from test_gpu_batch import replicas
    reps = replicas(seed=45)
    counts = [len(qq) for (_, _, qq) in reps]
    n = sum(counts)

    def plans(tuning):
        return [MSM(box=L, periodic=True, cutoff=6.0, spacing=1.5, order=3, splitting=2, precision="mixed",
                    max_atoms=len(qq), tuning=tuning) for (L, _, qq) in reps]

    fp = plans(FFT)
    assert all(p.lattice_method == "fft" for p in fp)
    assert len({p.dims[0] for p in fp}) > 1
    pos = torch.tensor(np.vstack([p for (_, p, _) in reps]), device=dev)
    q = torch.tensor(np.concatenate([qq for (_, _, qq) in reps]), device=dev)
    E = torch.zeros(len(reps), dtype=torch.float64, device=dev)
    phi = torch.zeros(n, dtype=torch.float64, device=dev)
    F = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    gE = torch.linspace(0.5, 2.0, len(reps), dtype=torch.float64, device=dev)
    gp = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    gq = torch.zeros(n, dtype=torch.float64, device=dev)
    g = MSMBatch(fp).graph(pos, q, counts, E, phi, F, gE, gp, gq)
    g.launch()
    torch.cuda.synchronize()
    first = [t.clone() for t in (E, phi, F, gp, gq)]
    g.launch()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(first, (E, phi, F, gp, gq)))
    for p in fp:
        p.check_status()
    o = 0
    singles = {"fft": plans(FFT), "stencil": plans(STENCIL)}
    for r, c in enumerate(counts):
        for name, sp in singles.items():
            Es, phis, Fs = sp[r].eval(pos[o:o + c], q[o:o + c])
            torch.cuda.synchronize()
            assert abs(E[r].item() - Es.item()) <= 1e-6 * abs(Es.item()), (r, name)
            assert_atoms(F[o:o + c].cpu().numpy(), Fs.cpu().numpy(), 1e-5, (r, name))
            assert_atoms(phi[o:o + c].cpu().numpy(), phis.cpu().numpy(), 1e-6, (r, name))
            assert_atoms(gp[o:o + c].cpu().numpy(), -gE[r].item() * Fs.cpu().numpy(), 1e-5, (r, name))
            assert_atoms(gq[o:o + c].cpu().numpy(), gE[r].item() * phis.cpu().numpy(), 1e-5, (r, name))
        o += c
    L, p3, q3 = reps[4]
    ref = O.msm(O.Params(box=(L,) * 3, periodic=True, cutoff=6.0, spacing=1.5, order=3, split=2), p3, q3)
    s = sum(counts[:4])
    assert abs(E[4].item() - ref["E"]) <= 1e-6 * abs(ref["E"])
    assert_atoms(F[s:s + counts[4]].cpu().numpy(), ref["F"], 1e-5)
    g.close()


def test_fft_replicas64_full_size_graph(dev):
    """The 64-replica benchmark batch (5,352-49,767 atoms, a = 10, h = 2,
    cubic, mixed) with the FFT lattice: every replica's energy and forces from
    the graph against its own plan's evaluation, three replicas against the
    oracle on a 256-atom spatial subsample."""
    from paper_1402_7216_gb300 import MSM, MSMBatch
    from synth import replica_boxes
    reps = replica_boxes(64)
    counts = [len(qq) for (_, _, qq) in reps]
    n = sum(counts)
    plans = [MSM(box=L, periodic=True, cutoff=10.0, spacing=2.0, order=3, splitting=2, precision="mixed",
                 max_atoms=len(qq), tuning=FFT) for (L, _, qq) in reps]
    assert all(p.lattice_method == "fft" for p in plans)
    pos = torch.tensor(np.vstack([p for (_, p, _) in reps]), device=dev)
    q = torch.tensor(np.concatenate([qq for (_, _, qq) in reps]), device=dev)
    E = torch.zeros(64, dtype=torch.float64, device=dev)
    phi = torch.zeros(n, dtype=torch.float64, device=dev)
    F = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    g = MSMBatch(plans).graph(pos, q, counts, E, phi, F)
    g.launch()
    torch.cuda.synchronize()
    Eg, Fg, phig = E.cpu().numpy(), F.cpu().numpy(), phi.cpu().numpy()
    off = np.cumsum([0] + counts)
    for r, p in enumerate(plans):
        E1, _, F1 = p.eval(pos[off[r]:off[r + 1]], q[off[r]:off[r + 1]])
        torch.cuda.synchronize()
        p.check_status()
        assert abs(Eg[r] - E1.item()) <= 1e-6 * abs(E1.item()), r
        assert_atoms(Fg[off[r]:off[r + 1]], F1.cpu().numpy(), 1e-5, r)
    order = np.argsort(counts)
    for r in (order[0], order[32], order[-1]):
        L, p_r, q_r = reps[r]
        pick = spatial_subsample(p_r, L, 256, seed=int(r))
        ref = O.msm(O.Params(box=(L,) * 3, periodic=True, cutoff=10.0, spacing=2.0, order=3, split=2), p_r, q_r,
                    targets=pick)
        assert_atoms(Fg[off[r]:off[r + 1]][pick], ref["F"], 1e-5, r)
        assert_atoms(phig[off[r]:off[r + 1]][pick], ref["phi"], 1e-5, r)
    g.close()


def test_fft_takes_stencils_beyond_the_stencil_window(dev):
    """FP64 with 2a/h = 31 (a stencil 30 grid spacings in radius) is past the
    FP64 stencil kernel's shared-memory window (about 27): the periodic plan
    evaluates it by FFT and matches the oracle; the stencil form and the open
    box, which would need that kernel, stay UNSUPPORTED."""
    from paper_1402_7216_gb300 import MSMError
    cfg = dict(box=15.5, periodic=True, cutoff=6.0, spacing=0.4, order=3, split=2)
    pos, q = water(cfg, 46, 0.03)
    for bad in (dict(cfg, periodic=False), cfg):
        with pytest.raises(MSMError) as e:
            rect_plan(bad, "fp64", len(q), STENCIL)
        assert e.value.code == -2
    plan = rect_plan(cfg, "fp64", len(q), FFT)
    assert plan.lattice_method == "fft" and plan.dims[0] == (40, 40, 40)
    assert_close(gpu_eval(plan, pos, q, dev), O.msm(oparams(cfg), pos, q), "fp64", "wide stencil")
