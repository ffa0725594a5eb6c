"""Learned global-move proposal: tensor-core GEMM, network forward/backward and the exact MH move,
through the C ABI, against plain FP32/FP64 references."""
import ctypes

import numpy as np
import pytest

import paper_2511_13508_gb300 as pkg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()


@pytest.mark.parametrize("batch,M,N,K", [(1, 128, 256, 64), (3, 200, 256, 192), (2, 77, 192, 256),
                                         (1, 300, 64, 520), (2, 129, 16, 24), (1, 512, 256, 512)])
def test_tcgen05_gemm_matches_fp32_reference(batch, M, N, K):
    import torch
    g = torch.Generator(device="cuda").manual_seed(M * N + K)
    A = torch.randn(batch, M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(batch, N, K, device="cuda", generator=g).to(torch.bfloat16)
    D = torch.full((batch, M, N), float("nan"), device="cuda", dtype=torch.float32)
    L = pkg.lib()
    L.pt_gemm_bf16.argtypes = [ctypes.c_int] * 4 + [ctypes.c_void_p] * 4
    s = torch.cuda.current_stream()
    rc = L.pt_gemm_bf16(batch, M, N, K, A.data_ptr(), B.data_ptr(), D.data_ptr(), s.cuda_stream)
    assert rc == 0, L.pt_last_error(None)
    torch.cuda.synchronize()
    ref = torch.bmm(A.float(), B.float().transpose(1, 2))
    err = (D - ref).abs().max().item()
    assert err <= 1e-4 * ref.abs().max().item() + 1e-4, err
