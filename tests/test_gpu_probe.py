"""bench.py's FP32 FMA throughput probe (fma_probe.cu, the roofline
denominator of the ALU-bound kernels): both forms run, their chains stay
finite, and invalid arguments are refused."""
import ctypes

import pytest
import torch

pytestmark = pytest.mark.gpu


def test_fma_probe_runs_and_rejects_bad_arguments():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from bench import load_fma_probe
    L = load_fma_probe()
    dev = torch.device("cuda:0")
    outs = []
    for packed in (1, 0):
        out = torch.empty(4 * 256, dtype=torch.float32, device=dev)
        rc = L.fma_probe(packed, 1000, 4, ctypes.c_void_p(out.data_ptr()),
                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        outs.append(out)
    assert L.fma_probe(1, -1, 4, ctypes.c_void_p(outs[0].data_ptr()), None) == -1
    assert L.fma_probe(1, 10, 0, ctypes.c_void_p(outs[0].data_ptr()), None) == -1
