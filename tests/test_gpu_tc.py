"""Tensor-core primitive (tcgen05.mma BF16 -> FP32 in tensor memory) against a
float64 matmul of the same BF16 values."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2505_08222_gb300 as ut  # noqa: E402


@pytest.mark.parametrize("M,N,K", [(128, 16, 16), (128, 64, 64), (256, 128, 128), (300, 256, 256), (1, 192, 96),
                                   (130, 48, 32)])
def test_tc_gemm_matches_float64(M, N, K):
    g = torch.Generator().manual_seed(M * 7 + N + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    C = ut.tc_gemm(A.cuda(), B.cuda()).cpu().double()
    ref = A.double() @ B.double().T
    # exact products of BF16 values, FP32 accumulation over K terms
    tol = 1e-5 * K * (A.double().abs() @ B.double().abs().T) + 1e-6
    assert torch.all((C - ref).abs() <= tol), float((C - ref).abs().max())


def test_tc_gemm_rejects_bad_shapes():
    A = torch.zeros(128, 20, dtype=torch.bfloat16, device="cuda")
    B = torch.zeros(16, 20, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(ut.UtError):
        ut.tc_gemm(A, B)
