"""Tensor-core (tcgen05) BF16 GEMM against a plain PyTorch FP32 reference.

The products of BF16 inputs are exact in FP32, so the only difference is the
FP32 accumulation order: relative error ~1e-6 of the row scale."""
import numpy as np
import pytest

from paper_1211_0126_gb300 import tsm

pytestmark = pytest.mark.gpu

CASES = [(128, 16, 64), (300, 96, 864), (257, 16, 72), (1000, 192, 128), (384, 300, 64), (5, 48, 8),
         (2000, 96, 1728)]


@pytest.mark.parametrize("m,n,k", CASES)
def test_umma_gemm_matches_fp32_reference(libtsm, m, n, k):
    import torch
    g = torch.Generator(device="cuda").manual_seed(m * 1000 + n + k)
    A = torch.randn(m, k, generator=g, device="cuda").to(torch.bfloat16)
    B = torch.randn(n, k, generator=g, device="cuda").to(torch.bfloat16)
    C = torch.full((m, n), float("nan"), device="cuda")
    tsm.tsm_umma_gemm(A, B, C)
    ref = A.float() @ B.float().T
    err = (C - ref).abs().max().item()
    scale = ref.abs().max().item()
    assert err <= 2e-5 * scale * max(1.0, np.sqrt(k / 64)), (err, scale)
    # accumulate mode: C += A B^T
    tsm.tsm_umma_gemm(A, B, C, beta=1)
    assert (C - 2 * ref).abs().max().item() <= 4e-5 * scale * max(1.0, np.sqrt(k / 64))
