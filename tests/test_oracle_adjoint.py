"""Pins of the oracle's deconvolution gradient.  CPU only.

* central finite differences of L(F) = ||T full(F) - g||^2 on core entries
  (FP64; L is quadratic in each core entry, so the central difference is
  exact up to rounding);
* the adjoint identity <T x, y> = <x, T y> of the dense operator;
* the partial products used by the chain rule reproduce full(F).
"""
import numpy as np
import pytest

from oracle import qtt as Q, conv as C, pipeline as P


def _cores(rng, d, r, cplx=False):
    ranks = [1] + [min(r, 2 ** k, 2 ** (d - k)) for k in range(1, d)] + [1]
    out = []
    for k in range(d):
        c = rng.standard_normal((ranks[k], 2, ranks[k + 1]))
        if cplx:
            c = c + 1j * rng.standard_normal(c.shape)
        out.append(c / np.sqrt(2 * ranks[k]))
    return out


@pytest.mark.parametrize("shape", [(256,), (16, 16)])
def test_core_grads_match_finite_differences(shape):
    rng = np.random.default_rng(3)
    d = int(np.log2(np.prod(shape)))
    cores = _cores(rng, d, 4)
    g = rng.standard_normal(shape)
    B = 6.0
    w = P.deconv_dense_grad(cores, shape, B, g)
    wq = w if len(shape) == 1 else Q.image_to_qtt_vector(w)
    grads = P.core_grads(cores, wq)
    h = 1e-3
    for k in (0, d // 2, d - 1):
        for idx in [(0, 0, 0), tuple(s - 1 for s in cores[k].shape)]:
            cp = [c.copy() for c in cores]
            cm = [c.copy() for c in cores]
            cp[k][idx] += h
            cm[k][idx] -= h
            fd = (P.deconv_loss(cp, shape, B, g) - P.deconv_loss(cm, shape, B, g)) / (2 * h)
            assert abs(fd - grads[k][idx].real) <= 1e-8 * (1 + abs(fd))


def test_core_grads_complex_wirtinger():
    # complex cores: 2 dL/dconj(F) -> real part by FD on Re, imag part by FD on Im
    rng = np.random.default_rng(4)
    d, shape = 7, (128,)
    cores = _cores(rng, d, 3, cplx=True)
    g = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    w = P.deconv_dense_grad(cores, shape, 5.0, g)
    grads = P.core_grads(cores, w)
    h = 1e-3
    k, idx = 3, (1, 0, 2)
    for part, unit in ((0, 1.0), (1, 1j)):
        cp = [c.copy() for c in cores]
        cm = [c.copy() for c in cores]
        cp[k][idx] += h * unit
        cm[k][idx] -= h * unit
        fd = (P.deconv_loss(cp, shape, 5.0, g) - P.deconv_loss(cm, shape, 5.0, g)) / (2 * h)
        val = grads[k][idx].real if part == 0 else grads[k][idx].imag
        assert abs(fd - val) <= 1e-8 * (1 + abs(fd))


def test_dense_adjoint_identity():
    rng = np.random.default_rng(5)
    n = 512
    taps = C.sinc_taps(n, 20.0)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    y = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    lhs = np.vdot(C.conv_fft(x, taps), y)
    rhs = np.vdot(x, C.conv_fft(y, taps))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_partials_reproduce_full():
    rng = np.random.default_rng(6)
    cores = _cores(rng, 8, 3, cplx=True)
    f = Q.full(cores)
    for k in range(1, 8):
        Lp = P._left_partial(cores[:k])
        Rp = P._right_partial(cores[k:])
        assert np.allclose((Lp @ Rp).reshape(-1, order='F'), f, atol=1e-13)
