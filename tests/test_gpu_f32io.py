"""msm_eval_f32io / msm_eval_backward_f32io: FP32 positions, charges and
per-atom outputs through the same plan.

On inputs that FP32 represents exactly, both entry points feed the kernels the
same numbers (the mixed plan splits an FP64 coordinate into hi + lo floats, and
a float-representable one has lo = 0), so the two agree up to the order of
atomic additions and the final rounding of the outputs to FP32:
  energy rel 1e-7, force / potential / gradient rel-RMS 1e-6.
Against the FP64 oracle on the same rounded inputs the usual mixed-precision
tolerances hold (energy rel 1e-6, force rel-RMS 1e-5, potential rel-RMS 1e-6).
"""
import numpy as np
import pytest
import torch

import oracle as O
from conftest import assert_atoms, rel_rms
from synth import make_water_box

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_7216_gb300 import lib
    lib()
    return torch.device("cuda:0")


def rounded_box(box, periodic, seed):
    pos, q = make_water_box(box, 420, 3, 2, seed=seed, periodic=periodic)
    return pos.astype(np.float32).astype(np.float64), q.astype(np.float32).astype(np.float64)


def plan(cfg, precision, n):
    from paper_1402_7216_gb300 import MSM
    return MSM(box=cfg["box"], periodic=cfg["periodic"], cutoff=cfg["cutoff"], spacing=cfg["spacing"],
               order=cfg["order"], splitting=cfg["split"], precision=precision, max_atoms=n)


CFGS = [dict(name="per-quintic", box=24.0, periodic=True, cutoff=8.0, spacing=2.0, order=5, split=2),
        dict(name="open-cubic", box=24.0, periodic=False, cutoff=8.0, spacing=2.0, order=3, split=2)]


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("cfg", CFGS, ids=[c["name"] for c in CFGS])
def test_f32io_matches_f64io_and_oracle(cfg, precision, dev):
    pos, q = rounded_box(cfg["box"], cfg["periodic"], seed=61)
    p = plan(cfg, precision, len(q))
    E64, phi64, F64 = p.eval(torch.tensor(pos, device=dev), torch.tensor(q, device=dev))
    p32, q32 = torch.tensor(pos, dtype=torch.float32, device=dev), torch.tensor(q, dtype=torch.float32, device=dev)
    E32, phi32, F32 = p.eval_f32io(p32, q32)
    torch.cuda.synchronize()
    p.check_status()
    assert phi32.dtype == torch.float32 and F32.dtype == torch.float32 and E32.dtype == torch.float64
    assert abs(E32.item() - E64.item()) <= 1e-7 * abs(E64.item())
    assert_atoms(F32.double().cpu().numpy(), F64.cpu().numpy(), 1e-6)
    assert_atoms(phi32.double().cpu().numpy(), phi64.cpu().numpy(), 1e-6)
    b = cfg["box"]
    ref = O.msm(O.Params(box=(b, b, b), periodic=cfg["periodic"], cutoff=cfg["cutoff"], spacing=cfg["spacing"],
                         order=cfg["order"], split=cfg["split"]), pos, q)
    assert abs(E32.item() - ref["E"]) <= 1e-6 * abs(ref["E"])
    assert_atoms(F32.double().cpu().numpy(), ref["F"], 1e-5)
    assert_atoms(phi32.double().cpu().numpy(), ref["phi"], 1e-6)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_backward_f32io_matches_backward(precision, dev):
    cfg = CFGS[0]
    pos, q = rounded_box(cfg["box"], True, seed=62)
    p = plan(cfg, precision, len(q))
    g = torch.tensor(0.75, dtype=torch.float64, device=dev)
    p.eval(torch.tensor(pos, device=dev), torch.tensor(q, device=dev), want_phi=False, want_force=False)
    gp64, gq64 = p.backward(g)
    p.eval_f32io(torch.tensor(pos, dtype=torch.float32, device=dev), torch.tensor(q, dtype=torch.float32, device=dev),
                 want_phi=False, want_force=False)
    gp32, gq32 = p.backward(g)
    torch.cuda.synchronize()
    assert gp32.dtype == torch.float32 and gq32.dtype == torch.float32
    assert_atoms(gp32.double().cpu().numpy(), gp64.cpu().numpy(), 1e-6)
    assert_atoms(gq32.double().cpu().numpy(), gq64.cpu().numpy(), 1e-6)


def test_autograd_with_float32_tensors(dev):
    from paper_1402_7216_gb300 import MSMEnergy
    cfg = CFGS[0]
    pos, q = rounded_box(cfg["box"], True, seed=63)
    p = plan(cfg, "mixed", len(q))
    x = torch.tensor(pos, dtype=torch.float32, device=dev, requires_grad=True)
    c = torch.tensor(q, dtype=torch.float32, device=dev, requires_grad=True)
    E = MSMEnergy.apply(x, c, p)
    E.backward()
    _, phi, F = p.eval(torch.tensor(pos, device=dev), torch.tensor(q, device=dev))
    torch.cuda.synchronize()
    assert x.grad.dtype == torch.float32 and c.grad.dtype == torch.float32
    assert_atoms(-x.grad.double().cpu().numpy(), F.cpu().numpy(), 1e-6)
    assert_atoms(c.grad.double().cpu().numpy(), phi.cpu().numpy(), 1e-6)


def test_f32io_periodic_images_and_errors(dev):
    from paper_1402_7216_gb300 import MSMError
    cfg = CFGS[0]
    pos, q = rounded_box(cfg["box"], True, seed=64)
    pos = np.round(pos * 4096.0) / 4096.0  # so that pos + k L stays exact in FP32 below
    p = plan(cfg, "mixed", len(q))
    q32 = torch.tensor(q, dtype=torch.float32, device=dev)
    E0, _, F0 = p.eval_f32io(torch.tensor(pos, dtype=torch.float32, device=dev), q32)
    # whole-box shifts of some atoms (folded back on the device); positions on
    # a 2^-12 lattice keep pos + k L exact in FP32
    shift = np.zeros_like(pos)
    shift[::3, 0] = 24.0
    shift[1::3, 1] = -48.0
    shift[2::5, 2] = 72.0
    E1, _, F1 = p.eval_f32io(torch.tensor(pos + shift, dtype=torch.float32, device=dev), q32)
    torch.cuda.synchronize()
    p.check_status()
    assert abs(E1.item() - E0.item()) <= 1e-6 * abs(E0.item())
    assert_atoms(F1.double().cpu().numpy(), F0.double().cpu().numpy(), 1e-5)
    # device-detected errors through the FP32 entry point
    ocfg = CFGS[1]
    po = plan(ocfg, "mixed", 8)
    bad = torch.tensor([[1.0, 2.0, 3.0], [25.0, 1.0, 1.0]], dtype=torch.float32, device=dev)
    po.eval_f32io(bad, torch.tensor([1.0, -1.0], dtype=torch.float32, device=dev))
    assert po.status() == -4
    bad[1, 0] = float("inf")
    po.eval_f32io(bad, torch.tensor([1.0, -1.0], dtype=torch.float32, device=dev))
    assert po.status() == -5
    with pytest.raises(ValueError):
        po.eval(bad, torch.tensor([1.0, -1.0], dtype=torch.float64, device=dev))
    with pytest.raises(MSMError):
        po.eval_f32io(torch.zeros((9, 3), dtype=torch.float32, device=dev),
                      torch.zeros(9, dtype=torch.float32, device=dev))
