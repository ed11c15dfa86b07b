"""The FP32 FMA throughput probe behind the roofline denominators: both forms
run, their chains stay finite, and invalid arguments are refused."""
import ctypes

import pytest
import torch

pytestmark = pytest.mark.gpu


def test_fma_probe_runs_and_rejects_bad_arguments():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_7216_gb300 import lib
    dev = torch.device("cuda:0")
    outs = []
    for packed in (1, 0):
        out = torch.empty(4 * 256, dtype=torch.float32, device=dev)
        rc = lib().msm_fma_probe(packed, 1000, 4, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        outs.append(out)
    assert lib().msm_fma_probe(1, -1, 4, ctypes.c_void_p(outs[0].data_ptr()), None) == -1
    assert lib().msm_fma_probe(1, 10, 0, ctypes.c_void_p(outs[0].data_ptr()), None) == -1
