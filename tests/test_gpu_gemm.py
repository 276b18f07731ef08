"""The network's BF16 product on the tcgen05 tensor cores (tmr_gemm_bf16,
C = A B^T with FP32 accumulation in tensor memory) against an FP64 product of
the same BF16-rounded operands: every element within FP32 accumulation error
of its exact value, on shapes with tails in M, N and K and with row strides
wider than the rows; shapes outside the kernel's range are refused."""
import numpy as np
import pytest

from helpers import to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2302_13524_gb300 as tmr  # noqa: E402


def _check(M, N, K, pad_a=0, pad_b=0, seed=0):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    A = torch.randn((M, K + pad_a), generator=g, device="cuda").to(torch.bfloat16)[:, :K]
    B = torch.randn((N, K + pad_b), generator=g, device="cuda").to(torch.bfloat16)[:, :K]
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    tmr.tmr_gemm_bf16(A, B, C)
    a = to_np(A.float()).astype(np.float64)
    b = to_np(B.float()).astype(np.float64)
    ref = a @ b.T
    bound = 1e-5 * (np.abs(a) @ np.abs(b).T) + 1e-30
    err = np.abs(to_np(C).astype(np.float64) - ref)
    assert np.all(err <= bound), (M, N, K, float(np.max(err / bound)))


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 384, 512), (296, 264, 200), (1000, 136, 72),
                                   (640, 1024, 8192)])
def test_tc_gemm_matches_fp64(M, N, K):
    _check(M, N, K)


def test_tc_gemm_row_strides():
    _check(300, 200, 136, pad_a=24, pad_b=8, seed=3)


def test_tc_gemm_refuses_other_shapes():
    A = torch.zeros((100, 64), dtype=torch.bfloat16, device="cuda")
    B = torch.zeros((128, 64), dtype=torch.bfloat16, device="cuda")
    C = torch.zeros((100, 128), dtype=torch.float32, device="cuda")
    with pytest.raises(tmr.TMRError) as ei:  # M < 128
        tmr.tmr_gemm_bf16(A, B, C)
    assert ei.value.status == tmr.TMR_ERR_UNSUPPORTED
    A = torch.zeros((128, 60), dtype=torch.bfloat16, device="cuda")
    B = torch.zeros((128, 60), dtype=torch.bfloat16, device="cuda")
    C = torch.zeros((128, 128), dtype=torch.float32, device="cuda")
    with pytest.raises(tmr.TMRError) as ei:  # K not a multiple of 8, below 64
        tmr.tmr_gemm_bf16(A, B, C)
    assert ei.value.status == tmr.TMR_ERR_UNSUPPORTED
