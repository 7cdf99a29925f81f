"""QTT-FFT / QTT-iFFT and the QTT convolution of Alg. 2 through the C ABI
(complex64) against the oracle (oracle/qfft.py) on the same seeded inputs
(random cores, or arrays the library decomposes itself):

* one transform, truncated to R^_max: the full spectrum within 1e-5
  (relative, FP32), ranks within the cap;
* untruncated small transforms against numpy's fft / fft2 (1D, 2D plain,
  2D interleaved; 2D results in the transposed image's layout);
* QiFFT(QFFT(x)) = x; the Hadamard product = the entrywise product;
* Alg. 2 (max rank TT-SVD with R_max = 10, transforms with R^_max = 15) on a
  Sec. 7 example against the oracle's route on the same noisy input, each
  side with its own kernel samples (qtt_sinc_padded on the device, checked
  against the oracle's Sec. 2 padding);
* argument errors: a real handle, an interleaved layout with unequal axes.

The Alg. 2 parity bound is derived from the oracle's own conditioning: a
chain of 3d roundings capped at R^_max amplifies small perturbations of the
cores, so the test first measures how far the oracle's result moves when
every core is perturbed by a relative 1e-7 (about one FP32 rounding) before
each rounding, and allows ten times that spread (at least 1e-5).
"""
import numpy as np
import pytest

from oracle import conv as C, qfft as QF, qtt as Q
import synth

pytestmark = pytest.mark.gpu


def _random_qtt(rng, d, r):
    ranks = [1] + [min(r, 2 ** k, 2 ** (d - k)) for k in range(1, d)] + [1]
    return [(rng.standard_normal((ranks[k], 2, ranks[k + 1]))
             + 1j * rng.standard_normal((ranks[k], 2, ranks[k + 1]))) for k in range(d)]


def _handle(q, cores, shape_log2, interleave=False):
    return q.qtt_from_cores([c.astype(np.complex64) for c in cores], shape_log2, interleave)


def _full(q, t):
    return q.qtt_to_full(t).cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("d,rhat", [(10, 15), (14, 15), (12, 8)])
def test_fft_truncated_parity(qlib, d, rhat):
    rng = np.random.default_rng(d + rhat)
    cores = _random_qtt(rng, d, 6)
    for inverse in (False, True):
        t = qlib.qtt_fft(_handle(qlib, cores, [d]), inverse=inverse, rmax=rhat)
        assert max(t.ranks()) <= rhat
        ref = Q.full(QF.qtt_fft(cores, rmax=rhat, inverse=inverse))
        got = _full(qlib, t)
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("d", [2, 5, 9])
def test_fft_exact_is_numpy_fft(qlib, d):
    rng = np.random.default_rng(50 + d)
    cores = _random_qtt(rng, d, 4)
    x = Q.full(cores)
    got = _full(qlib, qlib.qtt_fft(_handle(qlib, cores, [d]), rmax=64))
    ref = np.fft.fft(x)
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("dy,dx,interleave", [(3, 4, False), (4, 4, True), (2, 5, False)])
def test_fft_2d_is_fft2_transposed(qlib, dy, dx, interleave):
    import torch
    rng = np.random.default_rng(7 * dx + dy)
    img = rng.standard_normal((2 ** dy, 2 ** dx)) + 1j * rng.standard_normal((2 ** dy, 2 ** dx))
    # the library's own TT-SVD at full rank (exact) builds the input handle
    x = qlib.qtt_decompose(torch.from_numpy(img.astype(np.complex64)).cuda(), 0.0, 0, refine=True,
                           interleave=interleave)
    t = qlib.qtt_fft(x, rmax=64)
    assert t.shape == (2 ** dx, 2 ** dy)
    got = _full(qlib, t)
    ref = np.fft.fft2(img).T
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
    back = _full(qlib, qlib.qtt_fft(t, inverse=True, rmax=64))
    assert np.linalg.norm(back - img) <= 1e-5 * np.linalg.norm(img)


def test_round_trip(qlib):
    rng = np.random.default_rng(3)
    d = 16
    cores = _random_qtt(rng, d, 5)
    x = Q.full(cores)
    t = _handle(qlib, cores, [d])
    back = _full(qlib, qlib.qtt_fft(qlib.qtt_fft(t, rmax=32), inverse=True, rmax=32))
    assert np.linalg.norm(back - x) <= 1e-5 * np.linalg.norm(x)


@pytest.mark.parametrize("dtype", [np.float64, np.complex64])
def test_hadamard(qlib, dtype):
    rng = np.random.default_rng(9)
    d = 11
    A = _random_qtt(rng, d, 4)
    B = _random_qtt(rng, d, 3)
    if dtype == np.float64:
        A = [a.real.copy() for a in A]
        B = [b.real.copy() for b in B]
    ha = qlib.qtt_from_cores([a.astype(dtype) for a in A], [d])
    hb = qlib.qtt_from_cores([b.astype(dtype) for b in B], [d])
    z = qlib.qtt_hadamard(ha, hb)
    assert z.ranks() == [x * y for x, y in zip(Q.ranks_of(A), Q.ranks_of(B))]
    got = qlib.qtt_to_full(z).cpu().numpy()
    ref = Q.full(A) * Q.full(B)
    tol = 1e-12 if dtype == np.float64 else 1e-5
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)


@pytest.mark.parametrize("example,K", [(1, 14), (2, 14)])
def test_alg2_example_parity(qlib, example, K):
    """Alg. 2 on a Sec. 7 example at 2^K: the CUDA path (qtt_decompose with
    R_max = 10, qtt_conv_fft with R^_max = 15) against the oracle's route on
    the same noisy input, within ten times the oracle's own spread under
    FP32-sized perturbations of every stage (at least 1e-5)."""
    import torch
    noisy, clean, N, B = synth.paper_example_1d(example, K, synth.config_rng(5, sub=example))
    n = 2 ** K
    g = QF.padded_kernel(C.sinc_taps(n, B), N, n)
    ref = QF.conv_qtt_fft(noisy, g, 10, 15)
    tol = max(1e-5, 10.0 * QF.conv_qtt_fft_spread(noisy, g, 10, 15, ref))
    g_dev = qlib.qtt_sinc_padded(K, N, B)               # the library's own kernel samples
    F = qlib.qtt_decompose(torch.from_numpy(noisy.astype(np.complex64)).cuda(), 0.0, 10, refine=True)
    G = qlib.qtt_decompose(g_dev, 0.0, 10, refine=True)
    got = _full(qlib, qlib.qtt_conv_fft(F, G, rhat=15))
    assert tol <= 1e-4
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)


@pytest.mark.parametrize("K,B,normalize", [(8, 64.0, True), (12, 1024.0, True), (10, 37.5, False)])
def test_sinc_padded(qlib, K, B, normalize):
    import torch
    n = 2 ** K
    N = 2 ** (K - 1) - 1
    ref = QF.padded_kernel(C.sinc_taps(n, B, normalize), N, n)
    g64 = qlib.qtt_sinc_padded(K, N, B, normalize, dtype=torch.float64).cpu().numpy()
    assert np.abs(g64 - ref).max() <= 1e-13 * np.abs(ref).max()
    g32 = qlib.qtt_sinc_padded(K, N, B, normalize).cpu().numpy()
    assert np.abs(g32.imag).max() == 0.0
    assert np.abs(g32.real - ref).max() <= 1e-6 * np.abs(ref).max()
    with pytest.raises(qlib.QTTError):
        qlib.qtt_sinc_padded(K, N + 1, B)


def test_argument_errors(qlib):
    rng = np.random.default_rng(1)
    real = qlib.qtt_from_cores([c.real.copy() for c in _random_qtt(rng, 6, 2)], [6])
    with pytest.raises(qlib.QTTError):
        qlib.qtt_fft(real)
    inter = _handle(qlib, _random_qtt(rng, 5, 2), [2, 3], interleave=True)
    with pytest.raises(qlib.QTTError):
        qlib.qtt_fft(inter)
    other = _handle(qlib, _random_qtt(rng, 5, 2), [5])
    with pytest.raises(qlib.QTTError):
        qlib.qtt_hadamard(inter, other)
