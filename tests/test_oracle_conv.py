"""Pins of the oracle's convolution definitions (Sec. 2, Eq. dconv; Eq. GAF).

CPU only.  Independent references: numpy.convolve (the Remark after Eq. dconv
identifies the discrete convolution with a 'same'-shaped convn times h^D),
explicit Python loops, closed forms of the sinc kernel.
"""
import numpy as np
import pytest

from oracle import conv as C


@pytest.mark.parametrize("n", [16, 32, 64, 128, 256])
def test_direct_equals_numpy_convolve(n):
    rng = np.random.default_rng(n)
    f = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    taps = C.sinc_taps(n, B=5.0, normalize=True)
    ref = np.convolve(f, taps)[n - 1:2 * n - 1]       # 'same' part of the full convolution
    assert np.allclose(C.conv_direct(f, taps), ref, rtol=0, atol=1e-14 * np.abs(ref).max())
    if n <= 64:
        assert np.allclose(C.conv_direct_loops(f, taps), ref, rtol=0, atol=1e-14 * np.abs(ref).max())


def test_fft_equals_direct_sums_large():
    n = 2 ** 14
    rng = np.random.default_rng(7)
    f = rng.standard_normal(n)
    taps = C.sinc_taps(n, B=300.0)
    out = C.conv_fft(f, taps)
    idx = rng.choice(n, 1024, replace=False)
    for j in idx:
        i = np.arange(n)
        direct = np.sum(f * taps[j - i + n - 1])
        assert abs(out[j] - direct) <= 1e-12 * np.abs(f).sum() * np.abs(taps).max()


def test_delta_input_gives_kernel_samples():
    # f = e_i  ->  I_j = h g((j - i) h): a closed form of the sinc kernel
    n, B, i0 = 128, 12.0, 37
    f = np.zeros(n)
    f[i0] = 1.0
    out = C.conv_direct(f, C.sinc_taps(n, B, normalize=False))
    h = 1.0 / n
    for j in range(n):
        u = np.pi * B * (j - i0) * h
        g = 1.0 if j == i0 else np.sin(u) / u
        assert abs(out[j] - h * g) <= 1e-15


def test_sinc_zeros_and_unit_mass():
    n, B = 1024, 16.0           # zeros of sinc(pi B x) at x = k / B -> m = k n / B = 64 k
    taps = C.sinc_taps(n, B, normalize=False)
    for k in range(1, 10):
        assert abs(taps[64 * k + n - 1]) < 1e-18
        assert abs(taps[-64 * k + n - 1]) < 1e-18
    assert abs(taps[n - 1] - 1.0 / n) < 1e-18                 # h * sinc(0)
    tn = C.sinc_taps(n, B, normalize=True)
    assert abs(tn.sum() - 1.0) < 1e-12                         # normalised: unit discrete mass
    assert np.allclose(tn, taps / taps.sum(), rtol=1e-14, atol=0)


def test_linearity_and_symmetry():
    n = 64
    rng = np.random.default_rng(3)
    taps = C.sinc_taps(n, 7.0)
    T = C.toeplitz_dense(taps)
    assert np.allclose(T, T.T)                                 # even kernel
    f, g = rng.standard_normal(n), rng.standard_normal(n)
    assert np.allclose(C.conv_direct(2 * f - 3 * g, taps),
                       2 * C.conv_direct(f, taps) - 3 * C.conv_direct(g, taps))


def test_2d_separable_equals_four_loops():
    ny, nx = 8, 16
    rng = np.random.default_rng(5)
    F = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    tx, ty = C.sinc_taps(nx, 3.0), C.sinc_taps(ny, 2.0)
    ref = np.zeros((ny, nx), dtype=complex)
    for y in range(ny):
        for x in range(nx):
            s = 0
            for yy in range(ny):
                for xx in range(nx):
                    s += F[yy, xx] * ty[y - yy + ny - 1] * tx[x - xx + nx - 1]
            ref[y, x] = s
    assert np.allclose(C.conv2d_separable(F, tx, ty), ref, atol=1e-14)
    assert np.allclose(C.conv2d_fft(F, tx, ty), ref, atol=1e-13)


def test_rel_l2_definition():
    a = np.array([3.0, 4.0])
    ref = np.array([0.0, 0.0 + 5.0])
    # ||a - ref|| / ||ref|| = sqrt(9 + 1) / 5
    assert abs(C.rel_l2(a, ref) - np.sqrt(10) / 5) < 1e-15
