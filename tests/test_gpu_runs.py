"""Target runs of the mixed-precision pair kernel (msm_tuning.pair_runs = 1):
a warp takes 32 consecutive atoms of the sorted order, across the cells of a
row, instead of one cell's atoms.  Every evaluation path that uses the pair
kernel (MSM, the cutoff method, Wolf summation, batched replicas) must match
the FP64 oracle as the one-cell kernel does, on boxes with the fewest cells
the runs accept (seven along a periodic x), open and sparse boxes, and cells
of more than 32 atoms (runs inside one cell); boxes with fewer cells fall
back to the one-cell kernel.

Tolerances (mixed path, as everywhere): energy rel 1e-6, force rel-RMS 1e-5,
potential rel-RMS 1e-6, each atom's error bounded by assert_atoms."""
import numpy as np
import pytest
import torch

import oracle as O
from conftest import assert_atoms
from synth import make_water_box, WORKLOADS

pytestmark = pytest.mark.gpu

TOL = dict(E=1e-6, F=1e-5, phi=1e-6)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_7216_gb300 import lib
    lib()
    return torch.device("cuda:0")


def msm_plan(cfg, n, runs, **tuning):
    from paper_1402_7216_gb300 import MSM
    return MSM(box=cfg["box"], periodic=cfg["periodic"], cutoff=cfg["cutoff"], spacing=cfg["spacing"],
               levels=cfg.get("levels", 0), order=cfg["order"], splitting=cfg["split"], precision="mixed",
               max_atoms=max(n, 1), tuning=dict(tuning, pair_runs=1 if runs else 2))


def check(got, ref, what=""):
    E, phi, F = got
    assert abs(E - ref["E"]) <= TOL["E"] * abs(ref["E"]), (what, E, ref["E"])
    assert_atoms(F, ref["F"], TOL["F"], what)
    assert_atoms(phi, ref["phi"], TOL["phi"], what)


def evaluate(fn, pos, q, dev, *args):
    E, phi, F = fn(torch.tensor(pos, device=dev), torch.tensor(q, device=dev), *args)
    torch.cuda.synchronize()
    return E.item(), phi.cpu().numpy(), F.cpu().numpy()


CASES = [
    # seven cells along x, the fewest a periodic plan takes runs with
    dict(name="periodic-7-cells", box=43.4, periodic=True, cutoff=12.0, spacing=2.0, order=3, split=2,
         waters=2700, ions=2),
    dict(name="water23k", box=62.2, periodic=True, cutoff=10.0, spacing=2.0, order=3, split=2, workload="water23k"),
    dict(name="water3k-open", box=30.0, periodic=False, cutoff=12.0, spacing=2.5, order=3, split=1,
         workload="water3k_open"),
    # sparse open box: cells of ~20 atoms, neighbour rows of +-1 cell
    dict(name="open-sparse", box=60.0, periodic=False, cutoff=9.0, spacing=2.0, order=5, split=2, waters=1500,
         ions=0),
    # cells of ~48 atoms (eight along x): runs inside one cell, two per cell
    dict(name="dense-cells", box=62.2, periodic=True, cutoff=10.0, spacing=2.0, order=3, split=3,
         workload="water23k", tuning=dict(cell_fill=48)),
]


def system(cfg):
    if "workload" in cfg:
        return WORKLOADS[cfg["workload"]].make()
    return make_water_box(cfg["box"], cfg["waters"], cfg["ions"], cfg["ions"], seed=61, periodic=cfg["periodic"])


def oparams(cfg):
    return O.Params(box=(cfg["box"],) * 3, periodic=cfg["periodic"], cutoff=cfg["cutoff"], spacing=cfg["spacing"],
                    levels=cfg.get("levels", 0), order=cfg["order"], split=cfg["split"])


@pytest.mark.parametrize("cfg", CASES, ids=[c["name"] for c in CASES])
def test_runs_match_oracle(cfg, dev):
    pos, q = system(cfg)
    ref = O.msm(oparams(cfg), pos, q)
    plan = msm_plan(cfg, len(q), True, **cfg.get("tuning", {}))
    got = evaluate(plan.eval, pos, q, dev)
    plan.check_status()
    check(got, ref, cfg["name"])
    # reproducible to the bit, and within rounding of the one-cell kernel
    again = evaluate(plan.eval, pos, q, dev)
    assert again[0] == got[0] and np.array_equal(again[2], got[2]) and np.array_equal(again[1], got[1])
    cells = evaluate(msm_plan(cfg, len(q), False, **cfg.get("tuning", {})).eval, pos, q, dev)
    assert_atoms(got[2], cells[2], 1e-5, cfg["name"])


def test_runs_fall_back_to_cells_below_seven_cells(dev):
    # 37 A with a = 12: six cells along x, too few for a periodic row of seven
    cfg = dict(box=37.0, periodic=True, cutoff=12.0, spacing=2.0, order=3, split=2)
    pos, q = make_water_box(37.0, 1700, 0, 0, seed=62, periodic=True)
    runs = evaluate(msm_plan(cfg, len(q), True).eval, pos, q, dev)
    cells = evaluate(msm_plan(cfg, len(q), False).eval, pos, q, dev)
    assert runs[0] == cells[0] and np.array_equal(runs[2], cells[2])
    check(runs, O.msm(oparams(cfg), pos, q))


def test_runs_cutoff_and_wolf_match_oracle(dev):
    from paper_1402_7216_gb300 import MSM
    box, a, alpha = 43.4, 12.0, 0.2
    pos, q = make_water_box(box, 2700, 2, 2, seed=63, periodic=True)
    P = O.Params(box=(box,) * 3, periodic=True, cutoff=a, spacing=2.0)
    plan = MSM(box=box, periodic=True, cutoff=a, spacing=2.0, order=3, splitting=2, precision="mixed",
               max_atoms=len(q), tuning={"pair_runs": 1})
    check(evaluate(plan.wolf_eval, pos, q, dev, alpha), O.wolf_sum(P, pos, q, alpha), "wolf")
    # the hard cutoff: pairs within rounding of r = a may go either way (both
    # valid), so the cutoff tests' comparison leaves those atoms out
    import test_gpu_cutoff as TC
    TC.check(evaluate(plan.cutoff_eval, pos, q, dev), O.cutoff_sum(P, pos, q), "mixed", pos, q, box, True, a)
    plan.check_status()


def test_runs_in_the_batch_graph(dev):
    from paper_1402_7216_gb300 import MSM, MSMBatch
    rng = np.random.default_rng(64)
    reps = []
    for n in (6000, 9000, 7500, 12000):  # 39-49 A: seven to nine cells of ~16 atoms along x
        nw = n // 3
        L = (3 * nw / 0.1) ** (1.0 / 3.0)
        pos, q = make_water_box(L, nw, 0, 0, seed=int(rng.integers(1 << 30)), periodic=True)
        reps.append((L, pos, q))

    def plans(runs):
        return [MSM(box=L, periodic=True, cutoff=6.0, spacing=1.5, order=3, splitting=2, precision="mixed",
                    max_atoms=len(q), tuning={"cell_fill": 16, "pair_runs": 1 if runs else 2}) for (L, _, q) in reps]

    counts = [len(q) for (_, _, q) in reps]
    n = sum(counts)
    pos = torch.tensor(np.vstack([p for (_, p, _) in reps]), device=dev)
    q = torch.tensor(np.concatenate([qq for (_, _, qq) in reps]), device=dev)
    E = torch.zeros(len(reps), dtype=torch.float64, device=dev)
    phi = torch.zeros(n, dtype=torch.float64, device=dev)
    F = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    gE = torch.ones(len(reps), dtype=torch.float64, device=dev)
    gp = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    gq = torch.zeros(n, dtype=torch.float64, device=dev)
    g = MSMBatch(plans(True)).graph(pos, q, counts, E, phi, F, gE, gp, gq)
    g.launch()
    E2, phi2, F2 = MSMBatch(plans(False)).eval(pos, q, counts)
    torch.cuda.synchronize()
    assert torch.allclose(E, E2, rtol=1e-6, atol=0)
    assert_atoms(F.cpu().numpy(), F2.cpu().numpy(), 1e-5)
    assert_atoms(phi.cpu().numpy(), phi2.cpu().numpy(), 1e-6)
    L, p0, q0 = reps[0]
    ref = O.msm(O.Params(box=(L,) * 3, periodic=True, cutoff=6.0, spacing=1.5, order=3, split=2), p0, q0)
    assert abs(E[0].item() - ref["E"]) <= 1e-6 * abs(ref["E"])
    assert_atoms(F[:counts[0]].cpu().numpy(), ref["F"], 1e-5)
    g.close()
