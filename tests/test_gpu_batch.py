"""Batched replicas (independent periodic water boxes of uneven size, each
with its own plan and grid geometry): msm_eval_batch, its adjoint and the
captured CUDA graph must give what one msm_eval per replica gives, and that
in turn matches the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from conftest import assert_atoms, rel_rms
from synth import make_water_box

pytestmark = pytest.mark.gpu


def replicas(seed=40, sizes=(1500, 900, 2400, 1200, 3000, 600)):
    rng = np.random.default_rng(seed)
    out = []
    for i, n in enumerate(sizes):
        nw = n // 3
        L = (3 * nw / 0.1) ** (1.0 / 3.0)
        pos, q = make_water_box(L, nw, 0, 0, seed=int(rng.integers(1 << 30)), periodic=True)
        out.append((L, pos, q))
    return out


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def make_plans(reps, precision, method=0):
    from paper_1402_7216_gb300 import MSM
    return [MSM(box=L, periodic=True, cutoff=6.0, spacing=1.5, order=3, splitting=2, precision=precision,
                max_atoms=len(q), tuning={"lattice_method": method}) for (L, _, q) in reps]


@pytest.mark.parametrize("method", [1, 2], ids=["stencil", "fft"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_single_evaluations(precision, method, dev):
    from paper_1402_7216_gb300 import MSMBatch
    reps = replicas()
    plans = make_plans(reps, precision, method)
    assert len({p.dims[0] for p in plans}) > 1          # uneven grids
    counts = [len(q) for (_, _, q) in reps]
    pos = torch.tensor(np.vstack([p for (_, p, _) in reps]), device=dev)
    q = torch.tensor(np.concatenate([qq for (_, _, qq) in reps]), device=dev)
    batch = MSMBatch(plans)
    E, phi, F = batch.eval(pos, q, counts)
    gE = torch.linspace(0.5, 2.0, len(reps), dtype=torch.float64, device=dev)
    gp, gq = batch.backward(gE, counts)
    torch.cuda.synchronize()
    tol = 1e-12 if precision == "fp64" else 1e-6
    o = 0
    singles = make_plans(reps, precision, method)
    for r, (L, p, qq) in enumerate(reps):
        n = len(qq)
        Es, phis, Fs = singles[r].eval(torch.tensor(p, device=dev), torch.tensor(qq, device=dev))
        torch.cuda.synchronize()
        assert abs(E[r].item() - Es.item()) <= tol * abs(Es.item())
        assert_atoms(F[o:o + n].cpu().numpy(), Fs.cpu().numpy(), (1e-12 if precision == "fp64" else 1e-5))
        # adjoint: dL/dq = g phi, dL/dr = -g F
        assert_atoms(gq[o:o + n].cpu().numpy(), gE[r].item() * phis.cpu().numpy(), 1e-5)
        assert_atoms(gp[o:o + n].cpu().numpy(), -gE[r].item() * Fs.cpu().numpy(), 1e-5)
        o += n
    # one replica against the oracle
    L, p, qq = reps[2]
    ref = O.msm(O.Params(box=(L,) * 3, periodic=True, cutoff=6.0, spacing=1.5, order=3, split=2), p, qq)
    s = sum(counts[:2])
    assert abs(E[2].item() - ref["E"]) <= (1e-10 if precision == "fp64" else 1e-6) * abs(ref["E"])
    assert_atoms(F[s:s + counts[2]].cpu().numpy(), ref["F"], (1e-9 if precision == "fp64" else 1e-5))


@pytest.mark.parametrize("method", [1, 2], ids=["stencil", "fft"])
def test_batch_graph_replays(method, dev):
    from paper_1402_7216_gb300 import MSMBatch
    reps = replicas(seed=41)
    plans = make_plans(reps, "mixed", method)
    counts = [len(q) for (_, _, q) in reps]
    n = sum(counts)
    pos = torch.tensor(np.vstack([p for (_, p, _) in reps]), device=dev)
    q = torch.tensor(np.concatenate([qq for (_, _, qq) in reps]), device=dev)
    E = torch.zeros(len(reps), dtype=torch.float64, device=dev)
    phi = torch.zeros(n, dtype=torch.float64, device=dev)
    F = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    gE = torch.linspace(0.5, 2.0, len(reps), dtype=torch.float64, device=dev)
    gp = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    gq = torch.zeros(n, dtype=torch.float64, device=dev)
    batch = MSMBatch(plans)
    # mixed plans of one order and splitting: every stage one launch over all replicas
    g = batch.graph(pos, q, counts, E, phi, F, gE, gp, gq)
    torch.cuda.synchronize()
    assert E.abs().sum().item() == 0.0                  # capturing runs nothing
    direct = MSMBatch(make_plans(reps, "mixed", method))
    E2, phi2, F2 = direct.eval(pos, q, counts)
    gscale = torch.cat([gE[r].expand(c) for r, c in enumerate(counts)])
    for _ in range(2):
        g.launch()
        torch.cuda.synchronize()
        assert torch.allclose(E, E2, rtol=1e-6, atol=0)
        assert_atoms(F.cpu().numpy(), F2.cpu().numpy(), 1e-5)
        assert_atoms(phi.cpu().numpy(), phi2.cpu().numpy(), 1e-6)
        assert_atoms(gp.cpu().numpy(), (-gscale[:, None] * F2).cpu().numpy(), 1e-5)
        assert_atoms(gq.cpu().numpy(), (gscale * phi2).cpu().numpy(), 1e-5)
        for p in plans:
            p.check_status()
    # one replica of the graph against the oracle
    L, p3, q3 = reps[3]
    ref = O.msm(O.Params(box=(L,) * 3, periodic=True, cutoff=6.0, spacing=1.5, order=3, split=2), p3, q3)
    s = sum(counts[:3])
    assert abs(E[3].item() - ref["E"]) <= 1e-6 * abs(ref["E"])
    assert_atoms(F[s:s + counts[3]].cpu().numpy(), ref["F"], 1e-5)
    # new inputs in the same buffers are picked up by the next replay
    pos.add_(0.37)
    g.launch()
    E3, _, _ = direct.eval(pos, q, counts)
    torch.cuda.synchronize()
    assert torch.allclose(E, E3, rtol=1e-6, atol=0)
    g.close()


def test_batch_graph_fallback_fp64(dev):
    """FP64 plans (or plans of different orders) are not batched kernel by
    kernel; their graph forks the replicas' own launch sequences instead."""
    from paper_1402_7216_gb300 import MSMBatch
    reps = replicas(seed=42, sizes=(900, 1500, 600))
    plans = make_plans(reps, "fp64")
    counts = [len(q) for (_, _, q) in reps]
    n = sum(counts)
    pos = torch.tensor(np.vstack([p for (_, p, _) in reps]), device=dev)
    q = torch.tensor(np.concatenate([qq for (_, _, qq) in reps]), device=dev)
    E = torch.zeros(len(reps), dtype=torch.float64, device=dev)
    F = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    g = MSMBatch(plans).graph(pos, q, counts, E, None, F)
    g.launch()
    E2, _, F2 = MSMBatch(make_plans(reps, "fp64")).eval(pos, q, counts)
    torch.cuda.synchronize()
    assert torch.allclose(E, E2, rtol=1e-12, atol=0)
    assert_atoms(F.cpu().numpy(), F2.cpu().numpy(), 1e-12)
    g.close()


def test_single_plan_graph_matches_eager_calls(dev):
    """A one-plan graph (forward + adjoint) replays the plan's own
    msm_eval / msm_eval_backward, and picks up changed inputs."""
    from paper_1402_7216_gb300 import MSM
    from synth import make_water_box
    L = 24.0
    pos, q = make_water_box(L, 400, 2, 2, seed=91, periodic=True)
    plan = MSM(box=L, periodic=True, cutoff=8.0, spacing=2.0, order=5, splitting=2, precision="mixed",
               max_atoms=len(q))
    tp, tq = torch.tensor(pos, device=dev), torch.tensor(q, device=dev)
    n = len(q)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    phi = torch.zeros(n, dtype=torch.float64, device=dev)
    F = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    gE = torch.ones(1, dtype=torch.float64, device=dev)
    gp = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    gq = torch.zeros(n, dtype=torch.float64, device=dev)
    g = plan.graph(tp, tq, E, phi, F, gE, gp, gq)
    for shift in (0.0, 0.37):
        tp.add_(shift)
        g.launch()
        torch.cuda.synchronize()
        E0, phi0, F0 = plan.eval(tp, tq)
        gp0, gq0 = plan.backward(torch.ones((), dtype=torch.float64, device=dev))
        torch.cuda.synchronize()
        plan.check_status()
        assert abs(E.item() - E0.item()) <= 1e-7 * abs(E0.item())
        for a, b in ((phi, phi0), (F, F0), (gp, gp0), (gq, gq0)):
            assert float(((a - b) ** 2).sum().sqrt() / (b ** 2).sum().sqrt()) < 1e-6
    g.close()


def test_replicas64_full_size_graph(dev):
    """The benchmark's 64-replica batch at full size (5,352-49,767 atoms each,
    a=10, h=2, cubic, mixed), replayed from its batch graph as the bench
    times it: every replica's energy, forces and adjoint against that
    replica's own msm_eval / msm_eval_backward, and three replicas (the
    smallest, a middle one, the largest) against the oracle on a spatial
    subsample of 256 atoms."""
    from paper_1402_7216_gb300 import MSM, MSMBatch
    from synth import replica_boxes, spatial_subsample
    reps = replica_boxes(64)
    counts = [len(q) for (_, _, q) in reps]
    n = sum(counts)
    # the stencil lattice here; the FFT form of the same graph is in test_gpu_fft.py
    plans = [MSM(box=L, periodic=True, cutoff=10.0, spacing=2.0, order=3, splitting=2, precision="mixed",
                 max_atoms=len(q), tuning={"lattice_method": 1}) for (L, _, q) in reps]
    pos = torch.tensor(np.vstack([p for (_, p, _) in reps]), device=dev)
    q = torch.tensor(np.concatenate([qq for (_, _, qq) in reps]), device=dev)
    E = torch.zeros(64, dtype=torch.float64, device=dev)
    phi = torch.zeros(n, dtype=torch.float64, device=dev)
    F = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    gE = torch.linspace(0.5, 2.0, 64, dtype=torch.float64, device=dev)
    gp = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    gq = torch.zeros(n, dtype=torch.float64, device=dev)
    g = MSMBatch(plans).graph(pos, q, counts, E, phi, F, gE, gp, gq)
    g.launch()
    g.launch()
    torch.cuda.synchronize()
    Eg, Fg, gpg, gqg = E.cpu().numpy(), F.cpu().numpy(), gp.cpu().numpy(), gq.cpu().numpy()
    o = 0
    for r, p in enumerate(plans):
        c = counts[r]
        E1, _, F1 = p.eval(pos[o:o + c], q[o:o + c])
        gp1, gq1 = p.backward(gE[r])
        torch.cuda.synchronize()
        p.check_status()
        assert abs(Eg[r] - E1.item()) <= 1e-6 * abs(E1.item()), r
        assert_atoms(Fg[o:o + c], F1.cpu().numpy(), 1e-5, r)
        assert_atoms(gpg[o:o + c], gp1.cpu().numpy(), 1e-5, r)
        assert_atoms(gqg[o:o + c], gq1.cpu().numpy(), 1e-5, r)
        o += c
    off = np.cumsum([0] + counts)
    order = np.argsort(counts)
    for r in (order[0], order[32], order[-1]):
        L, p_r, q_r = reps[r]
        pick = spatial_subsample(p_r, L, 256, seed=int(r))
        ref = O.msm(O.Params(box=(L,) * 3, periodic=True, cutoff=10.0, spacing=2.0, order=3, split=2), p_r, q_r,
                    targets=pick)
        assert_atoms(Fg[off[r]:off[r + 1]][pick], ref["F"], 1e-5, r)
        assert_atoms(phi.cpu().numpy()[off[r]:off[r + 1]][pick], ref["phi"], 1e-5, r)
    g.close()


def test_persistent_chains_match_per_pass_launches(dev):
    """batch_persistent = 1: the restriction and prolongation chains of the
    batched graph run as one cooperative launch each, with grid barriers
    between passes.  The element work is the same, in the same order, so the
    forward and the adjoint are bit-identical to the per-pass graph; two
    replays in a row and changed inputs give the same as well."""
    from paper_1402_7216_gb300 import MSM, MSMBatch
    reps = replicas()
    counts = [len(q) for (_, _, q) in reps]
    n = sum(counts)
    pos = torch.tensor(np.vstack([p for (_, p, _) in reps]), device=dev)
    q = torch.tensor(np.concatenate([qq for (_, _, qq) in reps]), device=dev)
    out = {}
    for persistent in (0, 1):
        plans = [MSM(box=L, periodic=True, cutoff=6.0, spacing=1.5, order=3, splitting=2, precision="mixed",
                     max_atoms=len(qq), tuning={"batch_persistent": persistent}) for (L, _, qq) in reps]
        E = torch.zeros(len(reps), dtype=torch.float64, device=dev)
        F = torch.zeros((n, 3), dtype=torch.float64, device=dev)
        gE = torch.full((len(reps),), 1.5, dtype=torch.float64, device=dev)
        gp = torch.zeros((n, 3), dtype=torch.float64, device=dev)
        gq = torch.zeros(n, dtype=torch.float64, device=dev)
        g = MSMBatch(plans).graph(pos, q, counts, E, None, F, gE, gp, gq)
        res = []
        for shift in (0.0, 0.0, 0.41):
            pos.add_(shift)
            g.launch()
            torch.cuda.synchronize()
            res.append([t.clone() for t in (E, F, gp, gq)])
        pos.sub_(0.41)
        for p in plans:
            p.check_status()
        g.close()
        assert all(torch.equal(a, b) for a, b in zip(res[0], res[1]))   # replays are reproducible
        out[persistent] = res
    for a, b in zip(out[0], out[1]):
        for x, y in zip(a, b):
            assert torch.equal(x, y)
