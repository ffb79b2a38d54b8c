"""Tensor-core (tcgen05) BF16 GEMM against a plain PyTorch FP32 reference.

The products of BF16 inputs are exact in FP32, so the only difference is the
FP32 accumulation order: relative error ~1e-6 of the row scale."""
import numpy as np
import pytest

from paper_1211_0126_gb300 import tsm

pytestmark = pytest.mark.gpu

CASES = [(128, 16, 64), (300, 96, 864), (257, 16, 72), (1000, 192, 128), (384, 300, 64), (5, 48, 8),
         (2000, 96, 1728), (700, 864, 96), (4096, 256, 512), (130, 224, 200)]


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


@pytest.mark.parametrize("m,n,k,splits", [(96, 72, 1536, 5), (576, 8, 4096, 16), (200, 864, 96, 1),
                                          (1000, 256, 640, 3)])
def test_umma_split_k_and_leading_dims(libtsm, m, n, k, splits):
    """Split-K partials sum to the product; operands read through row strides
    larger than K (a column window of wider matrices)."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(m + n + k + splits)
    Aw = torch.randn(m, k + 24, generator=g, device="cuda").to(torch.bfloat16)
    Bw = torch.randn(n, k + 40, generator=g, device="cuda").to(torch.bfloat16)
    A, B = Aw[:, 8:8 + k], Bw[:, 16:16 + k]
    C = torch.full((splits, m, n), float("nan"), device="cuda")
    used = tsm.tsm_umma_gemm_ex(A, B, C, splits=splits)
    assert 1 <= used <= splits
    got = C[:used].sum(0)
    ref = A.float() @ B.float().T
    scale = ref.abs().max().item()
    assert (got - ref).abs().max().item() <= 2e-5 * scale * max(1.0, np.sqrt(k / 64))
    # each partial is the product over its own K chunk
    chunk = -(-k // used)
    chunk = -(-chunk // 64) * 64
    for z in range(used):
        lo, hi = z * chunk, min(k, (z + 1) * chunk)
        pz = A[:, lo:hi].float() @ B[:, lo:hi].float().T
        assert (C[z] - pz).abs().max().item() <= 2e-5 * scale * max(1.0, np.sqrt(k / 64))


def test_umma_wait_timeout_reports_and_recovers(libtsm):
    """The bounded stage wait of the tensor-core kernel runs out on a stage
    that nothing fills (operand copies withheld by the fault-injection switch,
    nothing in flight): the call returns TSM_ERR_TIMEOUT, and the next call
    on the same device computes the product again."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(7)
    A = torch.randn(256, 256, generator=g, device="cuda").to(torch.bfloat16)
    B = torch.randn(64, 256, generator=g, device="cuda").to(torch.bfloat16)
    C = torch.zeros(256, 64, device="cuda")
    tsm.tsm_umma_inject_timeout(True)
    try:
        with pytest.raises(tsm.TsmError) as e:
            tsm.tsm_umma_gemm(A, B, C)
        assert e.value.status == -6   # TSM_ERR_TIMEOUT
    finally:
        tsm.tsm_umma_inject_timeout(False)
    C.fill_(float("nan"))
    tsm.tsm_umma_gemm(A, B, C)
    ref = A.float() @ B.float().T
    assert (C - ref).abs().max().item() <= 2e-5 * ref.abs().max().item() * 2
