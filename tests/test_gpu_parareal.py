"""Parareal (msm_parareal, Eq. parareal) with F = velocity Verlet on the MSM
force and G = velocity Verlet on the cutoff method, against the oracle's
parareal; the cutoff method's MD (msm_md_run, method "cutoff") and the
batched MD (msm_md_run_batch) against single runs.

Tolerances: FP64 plans 1e-9 A / 1e-9 on velocities after two iterations
(same arithmetic, other summation order); mixed fine plans 1e-5 A."""
import numpy as np
import pytest
import torch

from synth import make_ion_system

pytestmark = pytest.mark.gpu

L, A, H = 16.0, 6.0, 2.0


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def make_plan(n, precision, L=L, periodic=True, cutoff=A):
    from paper_1402_7216_gb300 import MSM
    return MSM(box=L, periodic=periodic, cutoff=cutoff, spacing=H, order=3, splitting=2, precision=precision,
               max_atoms=max(n, 1))


def oparams(L=L, periodic=True, cutoff=A):
    import oracle as O
    return O.Params(box=(L,) * 3, periodic=periodic, cutoff=cutoff, spacing=H, order=3, split=2)


def dev_tensors(dev, *arrays):
    return [torch.tensor(a, device=dev) for a in arrays]


def min_image(d, L=L):
    return d - L * np.round(d / L)


def system(n=48, seed=31):
    return make_ion_system(L, n, seed=seed, kind="plasma")


def test_md_cutoff_method_matches_oracle(dev):
    from oracle import cutoff_sum
    from oracle.md import velocity_verlet
    pos, q, im, vel = system()
    P = oparams()

    def force(r):
        out = cutoff_sum(P, r, q)
        return out["F"], out["E"]
    r_o, v_o, _, rec_o = velocity_verlet(force, pos, vel, im, 0.05, 15, wrap=lambda r: r - L * np.floor(r / L))
    plan = make_plan(len(q), "fp64")
    tp, tv, ti, tq = dev_tensors(dev, pos, vel, im, q)
    _, rec = plan.md_run(tp, tv, ti, tq, 0.05, 15, method="cutoff")
    torch.cuda.synchronize()
    assert np.abs(min_image(tp.cpu().numpy() - r_o)).max() < 1e-10
    assert np.abs(tv.cpu().numpy() - v_o).max() < 1e-10
    np.testing.assert_allclose(rec.cpu().numpy()[:, :3], rec_o[:, :3], rtol=1e-10)


def test_md_batch_matches_single_runs(dev):
    """Three systems of different sizes stepped together equal each stepped
    alone (FP64: same kernels, summation order aside)."""
    from paper_1402_7216_gb300 import MSMBatch
    systems = [system(n, seed) for n, seed in ((30, 41), (48, 42), (64, 43))]
    single = []
    for pos, q, im, vel in systems:
        plan = make_plan(len(q), "fp64")
        tp, tv, ti, tq = dev_tensors(dev, pos, vel, im, q)
        _, rec = plan.md_run(tp, tv, ti, tq, 0.05, 8)
        single.append((tp.cpu().numpy(), tv.cpu().numpy(), rec.cpu().numpy()))
    plans = [make_plan(len(s[1]), "fp64") for s in systems]
    cat = [np.concatenate([s[i] for s in systems]) for i in range(4)]
    tp, tq, ti, tv = dev_tensors(dev, cat[0], cat[1], cat[2], cat[3])
    counts = [len(s[1]) for s in systems]
    B = MSMBatch(plans)
    _, _, F = B.eval(tp, tq, counts, want_phi=False)
    rec = B.md_run(tp, tv, F, ti, tq, counts, 0.05, 8)
    torch.cuda.synchronize()
    off = np.cumsum([0] + counts)
    for r, (p1, v1, rec1) in enumerate(single):
        assert np.abs(min_image(tp.cpu().numpy()[off[r]:off[r + 1]] - p1)).max() < 1e-11
        assert np.abs(tv.cpu().numpy()[off[r]:off[r + 1]] - v1).max() < 1e-11
        np.testing.assert_allclose(rec.cpu().numpy()[r], rec1, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("precision,coarse_method", [("fp64", "cutoff"), ("mixed", "cutoff"), ("fp64", "msm")])
def test_parareal_matches_oracle(precision, coarse_method, dev):
    """G = the cutoff method (a = 6 A) or MSM with half the cutoff (a = 3 A)."""
    from paper_1402_7216_gb300 import parareal
    from oracle.parareal import md_parareal
    pos, q, im, vel = system()
    W, dtf, sf, dtc, sc = 4, 0.05, 5, 0.125, 2
    ac = A if coarse_method == "cutoff" else A / 2
    lam_o, hist_o, ch_o = md_parareal(oparams(), oparams(cutoff=ac), pos, vel, im, q, W, dtf, sf, dtc, sc, 2, 0.0,
                                      coarse_method=coarse_method)
    fine = [make_plan(len(q), precision) for _ in range(W)]
    coarse = make_plan(len(q), "fp64", cutoff=ac)
    tp, tv, ti, tq = dev_tensors(dev, pos, vel, im, q)
    lp, lv, iters, ch = parareal(fine, coarse, tp, tv, ti, tq, W, dtf, sf, dtc, sc, 2, 0.0,
                                 coarse_method=coarse_method)
    assert iters == 2
    tol = 1e-9 if precision == "fp64" else 1e-5
    for k in range(W + 1):
        assert np.abs(min_image(lp[k].cpu().numpy() - lam_o[k][0])).max() < tol
        assert np.abs(lv[k].cpu().numpy() - lam_o[k][1]).max() < tol * 10
    np.testing.assert_allclose(ch, np.array(ch_o), rtol=1e-3 if precision == "fp64" else 2e-2)


def test_parareal_converges_to_the_sequential_fine_run(dev):
    from paper_1402_7216_gb300 import parareal
    pos, q, im, vel = system(60, 33)
    W, dtf, sf = 5, 0.05, 4
    fine = [make_plan(len(q), "fp64") for _ in range(W)]
    tp, tv, ti, tq = dev_tensors(dev, pos, vel, im, q)
    lp, lv, iters, ch = parareal(fine, fine[0], tp, tv, ti, tq, W, dtf, sf, 0.1, 2, 20, 1e-9)
    assert iters <= W + 1
    assert ch[-1][0] <= 1e-9
    seq = make_plan(len(q), "fp64")
    sp, sv, si, sq = dev_tensors(dev, pos, vel, im, q)
    for k in range(1, W + 1):
        seq.md_run(sp, sv, si, sq, dtf, sf)      # F from the new positions (its own first force)
        assert np.abs(min_image(lp[k].cpu().numpy() - sp.cpu().numpy())).max() < 1e-8
        assert np.abs(lv[k].cpu().numpy() - sv.cpu().numpy()).max() < 1e-8


def test_mixed_parareal_reaches_the_sequential_fine_run_exactly(dev):
    """Mixed precision, G = MSM with half the cutoff: the mixed path is
    bit-reproducible, so the change per iteration falls to exactly 0 and
    after W iterations every time point equals the sequential fine run to
    the rounding of the correction g + (f - g) (1e-12; the noise floor of a
    path whose sums vary between runs was 1e-5 A)."""
    from paper_1402_7216_gb300 import MSM, parareal
    pos, q, im, vel = system(60, 35)
    W, dtf, sf = 4, 0.05, 4
    fine = [make_plan(len(q), "mixed") for _ in range(W)]
    coarse = MSM(box=L, periodic=True, cutoff=0.5 * A, spacing=H, order=3, splitting=2, precision="mixed",
                 max_atoms=len(q))
    tp, tv, ti, tq = dev_tensors(dev, pos, vel, im, q)
    lp, lv, iters, ch = parareal(fine, coarse, tp, tv, ti, tq, W, dtf, sf, 0.1, 2, W + 1, 0.0,
                                 coarse_method="msm")
    assert iters == W + 1 and ch[-1][0] == 0.0 and ch[-1][1] == 0.0
    seq = make_plan(len(q), "mixed")
    sp, sv, si, sq = dev_tensors(dev, pos, vel, im, q)
    for k in range(1, W + 1):
        seq.md_run(sp, sv, si, sq, dtf, sf)
        assert (lp[k] - sp).abs().max().item() <= 1e-12, k
        assert (lv[k] - sv).abs().max().item() <= 1e-12, k


def test_parareal_argument_errors(dev):
    from paper_1402_7216_gb300 import MSMError, parareal
    pos, q, im, vel = system(20, 34)
    tp, tv, ti, tq = dev_tensors(dev, pos, vel, im, q)
    a = make_plan(len(q), "mixed")
    with pytest.raises(MSMError) as e:
        parareal([a, a], a, tp, tv, ti, tq, 2, 0.05, 2, 0.1, 1, 1, 0.0)    # one plan twice in the window
    assert e.value.code == -1
    small = make_plan(8, "mixed")
    with pytest.raises(MSMError) as e:
        parareal([a], small, tp, tv, ti, tq, 1, 0.05, 2, 0.1, 1, 1, 0.0)   # coarse plan too small
    assert e.value.code == -9
    with pytest.raises(ValueError):
        parareal([a], a, tp, tv, ti, tq, 2, 0.05, 2, 0.1, 1, 1, 0.0)       # one plan per time point


def test_parareal_window_of_one_is_one_fine_propagation(dev):
    """W = 1: after one iteration lambda_1 = G + F - G = F(lambda_0)."""
    from paper_1402_7216_gb300 import parareal
    pos, q, im, vel = system(40, 35)
    fine = [make_plan(len(q), "fp64")]
    tp, tv, ti, tq = dev_tensors(dev, pos, vel, im, q)
    lp, lv, iters, ch = parareal(fine, make_plan(len(q), "fp64"), tp, tv, ti, tq, 1, 0.05, 6, 0.1, 3, 1, 0.0)
    assert iters == 1
    seq = make_plan(len(q), "fp64")
    sp, sv, si, sq = dev_tensors(dev, pos, vel, im, q)
    seq.md_run(sp, sv, si, sq, 0.05, 6)
    torch.cuda.synchronize()
    assert np.abs(min_image(lp[1].cpu().numpy() - sp.cpu().numpy())).max() < 1e-11
    assert np.abs(lv[1].cpu().numpy() - sv.cpu().numpy()).max() < 1e-11
    np.testing.assert_array_equal(lp[0].cpu().numpy(), pos)


def test_md_batch_mixed_with_records(dev):
    """The batched MD on mixed plans: each replica's records and trajectory
    match the same replica stepped alone (mixed tolerance).  16 steps: both
    run as one step replayed from a CUDA graph."""
    from paper_1402_7216_gb300 import MSMBatch
    systems = [system(n, seed) for n, seed in ((36, 51), (52, 52))]
    single = []
    for pos, q, im, vel in systems:
        plan = make_plan(len(q), "mixed")
        tp, tv, ti, tq = dev_tensors(dev, pos, vel, im, q)
        _, rec = plan.md_run(tp, tv, ti, tq, 0.05, 16)
        single.append((tp.cpu().numpy(), rec.cpu().numpy()))
    plans = [make_plan(len(s[1]), "mixed") for s in systems]
    cat = [np.concatenate([s[i] for s in systems]) for i in range(4)]
    tp, tq, ti, tv = dev_tensors(dev, cat[0], cat[1], cat[2], cat[3])
    counts = [len(s[1]) for s in systems]
    B = MSMBatch(plans)
    _, _, F = B.eval(tp, tq, counts, want_phi=False)
    rec = B.md_run(tp, tv, F, ti, tq, counts, 0.05, 16).cpu().numpy()
    off = np.cumsum([0] + counts)
    for r, (p1, rec1) in enumerate(single):
        assert np.abs(min_image(tp.cpu().numpy()[off[r]:off[r + 1]] - p1)).max() < 1e-6
        np.testing.assert_allclose(rec[r][:, :3], rec1[:, :3], rtol=1e-6)
