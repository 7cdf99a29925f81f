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


def _crand(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


@pytest.mark.parametrize("M,N,K,conj", [
    (64, 256, 8, False),      # one tile, one k chunk
    (100, 300, 77, True),     # ragged rows, columns and k; conjugated A
    (768, 384, 64, False),    # the range finder's widest panel
    (384, 768, 2000, True),   # long k: split, partials added with compensation
    (5, 3, 1, False),         # degenerate sizes inside one tile
])
def test_tc_cgemm_complex_3xtf32(qlib, M, N, K, conj):
    """Complex GEMM on the tensor cores against the FP64 product: FP32-level
    accuracy (the 3xTF32 split drops only the lo x lo term, ~2^-22 relative),
    element by element and in the norm."""
    import torch
    rng = np.random.default_rng(M * 7 + N + K)
    A = _crand(rng, M, K)
    B = _crand(rng, K, N)
    C, st = qlib.tc_cgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), conj_a=conj)
    assert st == 0
    got = C.cpu().numpy().astype(np.complex128)
    Ar = A.astype(np.complex128)
    ref = (Ar.conj() if conj else Ar) @ B.astype(np.complex128)
    # each chunk of 8 k is summed in the FP32 accumulator (error ~ u |chunk|,
    # u = 2^-24, |chunk| ~ 4 |a||b|) and the chunks are added with
    # compensation: for random signs the chunk errors add up like a random
    # walk, ~ u sqrt(k) |a||b| per element, i.e. ~u relative to |c|
    scale = np.sqrt(K) * np.abs(Ar).max() * np.abs(B).max()
    assert np.abs(got - ref).max() <= 4e-6 * scale
    u = 2.0 ** -24
    assert np.linalg.norm(got - ref) <= (1e-6 + 2 * u * np.sqrt(2 * K)) * np.linalg.norm(ref)


@pytest.mark.parametrize("K", [16, 4096])
def test_tc_cgemm_same_sign(qlib, K):
    """Positive operands with full 24-bit mantissas.  The round-to-nearest
    hi/lo split keeps every entry within 5e-7 of the FP64 product (a
    truncating split loses up to 2^-20 of every operand).  The tensor core's
    FP32 accumulator rounds one-signed, so a long uncompensated run would
    drift by ~k u of |C|; each 8-k chunk starts from zero in tensor memory
    and the chunk sums are added in FP32 registers with compensation, so the
    mean error stays a fraction of u |C| at any k."""
    import torch
    rng = np.random.default_rng(17 + K)
    M, N = 64, 256
    A = (rng.uniform(0.5, 1.0, (M, K)) + 1j * rng.uniform(0.5, 1.0, (M, K))).astype(np.complex64)
    B = (rng.uniform(0.5, 1.0, (K, N)) + 1j * rng.uniform(-0.1, 0.1, (K, N))).astype(np.complex64)
    C, st = qlib.tc_cgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    assert st == 0
    ref = A.astype(np.complex128) @ B.astype(np.complex128)
    err = C.cpu().numpy() - ref
    scale = np.abs(ref).max()
    assert np.abs(err).max() <= 5e-7 * scale
    assert abs(err.real.mean()) <= 3e-7 * scale


def test_tc_cgemm_exact_small_integers(qlib):
    """Gaussian integers with small parts are exact in TF32 and in the FP32
    accumulator: the tensor-core product equals the integer product."""
    import torch
    rng = np.random.default_rng(5)
    A = (rng.integers(-3, 4, (70, 40)) + 1j * rng.integers(-3, 4, (70, 40))).astype(np.complex64)
    B = (rng.integers(-3, 4, (40, 260)) + 1j * rng.integers(-3, 4, (40, 260))).astype(np.complex64)
    C, st = qlib.tc_cgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    assert st == 0
    assert np.array_equal(C.cpu().numpy(), A @ B)


def test_tc_cgemm_zero_k(qlib):
    import torch
    A = torch.zeros((10, 0), dtype=torch.complex64, device="cuda")
    B = torch.zeros((0, 7), dtype=torch.complex64, device="cuda")
    C, st = qlib.tc_cgemm(A, B)
    assert st == 0 and C.shape == (10, 7) and not C.abs().max().item()


@pytest.mark.parametrize("m,n,split", [
    (32, 1000, 1), (48, 777, 3), (64, 4096, 3), (100, 1003, 1), (128, 2050, 3), (128, 9, 1),
    (17, 64, 3),
])
def test_tc_gram_partials(qlib, m, n, split):
    """The sum of the tensor-core Gram partials against X X^H in FP64.  Both
    MMA arrangements are covered (2 m_pad <= 128: one MMA on [Y; Z]; above:
    Re G and Im G in two), ragged m and n, fewer columns than CTAs.  TF32
    operands (split 1) carry 2^-11 relative rounding each: the Gram entries
    are good to ~1e-3 of |X_a||X_b|; 3xTF32 to the FP32 level."""
    import torch
    rng = np.random.default_rng(m * 31 + n + split)
    X = _crand(rng, m, n)
    parts, st = qlib.tc_gram(torch.from_numpy(X).cuda(), split=split, max_parts=8)
    assert st == 0
    assert 1 <= parts.shape[0] <= 8
    G = parts.cpu().numpy().astype(np.complex128).sum(axis=0)
    Xr = X.astype(np.complex128)
    ref = Xr @ Xr.conj().T
    nrm = np.linalg.norm(Xr, axis=1)
    scale = np.outer(nrm, nrm)                  # |X_a| |X_b| bounds |G_ab|
    tol = 2e-3 if split == 1 else 2e-5
    assert np.all(np.abs(G - ref) <= tol * scale)
    # Hermitian up to the same rounding, and a real, positive diagonal
    assert np.all(np.abs(np.diag(G).imag) <= tol * nrm ** 2)
    assert np.all(np.diag(G).real > 0)
