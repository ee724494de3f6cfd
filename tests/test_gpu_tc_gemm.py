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


def _rows_scaled(rng, shape, spread):
    """Gaussian rows with row scales spread over 2^-spread .. 2^spread and
    entries spanning a few binades inside each row."""
    x = rng.standard_normal(shape) * np.exp2(rng.uniform(-3, 3, shape))
    return x * np.exp2(rng.integers(-spread, spread + 1, (shape[0], 1)))


@pytest.mark.parametrize("M,N,K", [(128, 32, 64), (256, 96, 512), (384, 160, 256)])
def test_ozaki_gemm_accuracy(M, N, K):
    """FP64 slice product: |C - A B^T| <= K 2^-31 max|A_i.| max|B_j.|.  Worst
    cases: the five slices leave each entry within 2^-35 max|row| (K 2^-34
    in the product), the dropped pairs i + j > 6 add at most K 2^-33 and the
    FP32 rounding of the level >= 4 accumulator about as much; a wrong slice,
    scale or lane mapping gives errors of order one."""
    import torch
    import paper_1708_02835_gb300 as egs
    rng = np.random.default_rng(7 * M + N + K)
    a, b = _rows_scaled(rng, (M, K), 20), _rows_scaled(rng, (N, K), 20)
    C = torch.full((M, N), float("nan"), dtype=torch.float64, device="cuda")
    egs.egs_ozaki_gemm_test(torch.as_tensor(a).cuda(), torch.as_tensor(b).cuda(), C)
    got = C.cpu().numpy()
    ref = a @ b.T
    bound = K * 2.0 ** -31 * np.outer(np.abs(a).max(axis=1), np.abs(b).max(axis=1))
    err = np.abs(got - ref)
    print("ozaki max err / bound %.3e" % float(np.max(err / bound)))
    assert np.all(np.isfinite(got))
    assert np.all(err <= bound)
    # two orders of magnitude more accurate than an FP32 product (35 against
    # 24 significant bits per entry)
    fp32 = (a.astype(np.float32) @ b.astype(np.float32).T).astype(np.float64)
    assert np.max(err / bound) < 1e-2 * np.max(np.abs(fp32 - ref) / bound)


def test_ozaki_gemm_exact_on_small_integers():
    """Entries that are integers in [-127, 127] fit the first slice exactly
    and the level-2 sums (<= 512 * 127^2 < 2^24) are exact in FP32: the
    product must equal the integer product bit for bit."""
    import torch
    import paper_1708_02835_gb300 as egs
    rng = np.random.default_rng(3)
    a = rng.integers(-127, 128, (256, 512)).astype(np.float64)
    b = rng.integers(-127, 128, (64, 512)).astype(np.float64)
    C = torch.empty((256, 64), dtype=torch.float64, device="cuda")
    egs.egs_ozaki_gemm_test(torch.as_tensor(a).cuda(), torch.as_tensor(b).cuda(), C)
    assert np.array_equal(C.cpu().numpy(), a @ b.T)


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_withheld_stage_times_out_and_the_context_stays_usable(prec):
    """Failure detection of the tensor-core pipeline: one ring stage is never
    loaded, so the MMA warp's bounded wait for it runs out (2 s), the kernel
    unwinds (its in-flight loads land, TMEM is freed) and the call returns
    EGS_ERR_TIMEOUT; the next call on the same context gives the right
    product."""
    import torch
    import paper_1708_02835_gb300 as egs
    M, N, K = 256, 512, 512
    rng = np.random.default_rng(7)
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
    C = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    with pytest.raises(egs.EgsError) as e:
        egs.egs_tc_gemm_test_withhold(A, B, C, prec, withhold_stage=3)
    assert e.value.status == egs.EGS_ERR_TIMEOUT
    C2 = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    egs.egs_tc_gemm_test(A, B, C2, prec)
    got = C2.cpu().numpy().astype(np.float64)
    ref = a64 @ b64.T
    assert np.all(np.abs(got - ref) <= 2.0 ** -16 * (np.abs(a64) @ np.abs(b64).T))
