"""The tcgen05 GEMM pipeline (TMA -> shared memory -> tcgen05.mma -> TMEM ->
tcgen05.ld) against an FP64 product of the same operand values.

Operands are generated exactly representable in the MMA input type (TF32:
10 explicit mantissa bits; BF16: 7), so every product is exact and only the
FP32 accumulation rounds: |C - A B^T| <= K 2^-24 sum_k |a_ik b_jk| bounds it;
the test uses 2^-16 sum_k |a_ik b_jk|, far below the O(1) errors a wrong
descriptor, swizzle or lane mapping produces.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _tf32_exact(rng, shape):
    a = rng.standard_normal(shape).astype(np.float32)
    u = a.view(np.uint32) & np.uint32(0xFFFFE000)
    return u.view(np.float32)


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (256, 512, 512), (384, 256, 1024)])
@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_tc_gemm_matches_fp64(M, N, K, prec):
    import torch
    import paper_1708_02835_gb300 as egs
    rng = np.random.default_rng(M + N + K)
    a = _tf32_exact(rng, (M, K))
    b = _tf32_exact(rng, (N, K))
    if prec == "bf16":
        A = torch.as_tensor(a).to(torch.bfloat16).cuda()
        B = torch.as_tensor(b).to(torch.bfloat16).cuda()
        a64 = A.float().cpu().numpy().astype(np.float64)
        b64 = B.float().cpu().numpy().astype(np.float64)
    else:
        A = torch.as_tensor(a).cuda()
        B = torch.as_tensor(b).cuda()
        a64, b64 = a.astype(np.float64), b.astype(np.float64)
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    egs.egs_tc_gemm_test(A, B, C, prec)
    got = C.cpu().numpy().astype(np.float64)
    ref = a64 @ b64.T
    scale = np.abs(a64) @ np.abs(b64).T
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref) <= 2.0 ** -16 * scale)
