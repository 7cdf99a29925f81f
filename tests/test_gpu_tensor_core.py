"""The tensor-core (tcgen05) MMA path through the C ABI's diagnostic entry:
TF32 operands in shared memory (canonical no-swizzle K-major layout), FP32
accumulation in tensor memory, read back by tcgen05.ld.  Checked against the
FP64 product at the TF32 rounding level (operands keep 10 mantissa bits:
relative error ~1e-3 per product, far below 1 and far above FP32's 1e-7)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,K", [(32, 8), (64, 32), (128, 64), (256, 16)])
def test_tc_gemm_tf32(qlib, N, K):
    import torch
    rng = np.random.default_rng(N + K)
    A = rng.standard_normal((128, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    C, err = qlib.tc_selftest(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    assert err == 0
    got = C.cpu().numpy().astype(np.float64)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel < 5e-3, rel
    # entry by entry: every element carries its own product, not a neighbour's
    assert np.abs(got - ref).max() <= 2e-2 * np.abs(ref).max()


def test_tc_gemm_exact_small_integers(qlib):
    """Small integers are exact in TF32 and in FP32 sums: the tensor-core
    product must equal the integer product exactly."""
    import torch
    rng = np.random.default_rng(3)
    A = rng.integers(-4, 5, (128, 16)).astype(np.float32)
    B = rng.integers(-4, 5, (64, 16)).astype(np.float32)
    C, err = qlib.tc_selftest(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    assert err == 0
    assert np.array_equal(C.cpu().numpy(), A @ B.T)
