"""Plain definitions of the discrete convolution (the oracle's "O1" level).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  float64/complex128.

Readings of the paper used here (where it is silent or garbled):
* Grid: midpoint rule of Sec. 2 on [0, 1], x_j = (j + 1/2) h, h = 1/N.
* Kernel: Eq. (GAF), g(x) = A sinc(pi x / Delta_x) with Delta_x = 1/B, i.e.
  g(x) = A sinc(pi B x), sinc(u) = sin(u)/u, sinc(0) = 1.  With
  ``normalize`` the constant A follows Eq. (sinc_kern1): the kernel is divided
  by its integral, taken here as the midpoint sum over the 2N-1 grid offsets
  m h, m = -(N-1)..N-1 (the discrete analogue of the integral over [-1, 1]),
  so A = 1 / (h sum_m sinc(pi B m h)).
* Convolution: Eq. (dconv), I_j = h^D sum_i f_i g((j - i) h): the kernel is
  evaluated at grid differences, so the same-size linear convolution is the
  Toeplitz matrix-vector product I = T f with T[j, i] = h g((j - i) h).  The
  printed centring offset (N/2 - 1) is not an integer for the paper's odd N;
  evaluating at grid differences is what the Remark after Eq. (dconv)
  (convn 'same' times h^D) computes for odd-length taps centred at 0.
* 2D: Eq. (sinc_kern2) is separable, so T = T_y (x) T_x and
  I[y, x] = sum T_y[y, y'] T_x[x, x'] F[y', x'].
"""
import numpy as np


def sinc_taps(n, B, normalize=True):
    """Toeplitz taps c[m + n - 1] = h g(m h), m = -(n-1)..n-1 (incl. h)."""
    h = 1.0 / n
    m = np.arange(-(n - 1), n, dtype=np.float64)
    # np.sinc(z) = sin(pi z)/(pi z), so sinc(pi B m h) = np.sinc(B m h).
    s = np.sinc(B * m * h)
    if normalize:
        A = 1.0 / (h * s.sum())
    else:
        A = 1.0
    return h * A * s


def toeplitz_dense(taps):
    """Dense T[j, i] = taps[j - i + n - 1]."""
    n = (len(taps) + 1) // 2
    j = np.arange(n)[:, None]
    i = np.arange(n)[None, :]
    return taps[j - i + n - 1]


def conv_direct_loops(f, taps):
    """Eq. (dconv) written as two Python loops (tiny inputs only)."""
    n = len(f)
    out = np.zeros(n, dtype=np.result_type(f, taps, np.float64))
    for j in range(n):
        acc = 0.0
        for i in range(n):
            acc += f[i] * taps[j - i + n - 1]
        out[j] = acc
    return out


def conv_direct(f, taps):
    """Eq. (dconv) as the dense Toeplitz matrix-vector product (n <= ~2^14)."""
    return toeplitz_dense(taps) @ f


def conv_fft(f, taps):
    """Linear convolution by zero-padded FFT (Sec. 2: pad to >= 2N-1).

    out[j] = sum_i f[i] taps[j - i + n - 1]; full linear convolution of f
    (length n) with taps (length 2n-1) has length 3n-2, of which entries
    n-1 .. 2n-2 are the ones wanted.
    """
    n = len(f)
    L = 1
    while L < 3 * n - 2:
        L *= 2
    F = np.fft.fft(f, L)
    G = np.fft.fft(taps, L)
    full = np.fft.ifft(F * G)
    out = full[n - 1:2 * n - 1]
    if not (np.iscomplexobj(f) or np.iscomplexobj(taps)):
        out = out.real
    return out


def conv2d_separable(F, taps_x, taps_y):
    """2D separable convolution I = T_y F T_x^T (dense Toeplitz factors)."""
    Tx = toeplitz_dense(taps_x)
    Ty = toeplitz_dense(taps_y)
    return Ty @ F @ Tx.T


def conv2d_fft(F, taps_x, taps_y):
    """2D separable convolution, each axis by zero-padded FFT."""
    out = np.apply_along_axis(conv_fft, 1, F, taps_x)
    out = np.apply_along_axis(conv_fft, 0, out, taps_y)
    return out


def rel_l2(a, ref):
    """E_2 of Eq. (err_conv); the 1/N^D factors cancel."""
    a = np.asarray(a)
    ref = np.asarray(ref)
    return float(np.linalg.norm((a - ref).ravel()) / np.linalg.norm(ref.ravel()))
