"""QTT-FFT, QTT-iFFT and the QTT convolution of Alg. 2 (test infrastructure:
the oracle; only tests/, __graft_entry__.smoke() and bench.py's CPU legs
use it).  complex128.

Sec. 4 names the QTT-FFT approximation of [DKS12] without giving its steps;
here it is the radix-2 decimation-in-frequency FFT written as one QTT
operator per bit, each followed by TT-rounding (Sec. 5 puts the truncated
SVD -- a rank cap R^_max, or a tolerance -- inside the QTT-FFT):

* the stage on bit p of an axis (its bits on any increasing set of modes,
  the least significant first) maps the pair (x_n, x_{n+2^(p-1)})
  of each size-2^p sub-transform to (x_n + x_{n+2^(p-1)},
  (x_n - x_{n+2^(p-1)}) w^n) with w = exp(-2 pi i / 2^p) (exp(+...) for
  the inverse) and n the lower p-1 bits: the butterfly [[1, 1], [1, -1]] on
  that mode and a diagonal twiddle w^(i_k 2^(k-1)) on each lower mode k,
  switched on by the new bit -- a TT operator of rank 2 (the switch travels
  down the bonds, through the other axis' modes in an interleaved chain),
  the identity on every other mode;
* after the K stages of an axis the mode of its bit j+1 holds output bit
  K-j (bit reversal); reversing the whole chain of cores restores the bit
  order of every axis and mirrors the axes' positions, so a 2D transform in
  the "x bits, then y bits" chain comes out in the "y bits, then x bits"
  chain (interleaved: y first); the inverse transform of a product (same
  chain for both factors) mirrors it back.

The Sec. 2 DFT convention: w_N = exp(-2 pi i / N), the inverse carries
1/N^D (numpy's fft/ifft).

``hadamard`` is the entrywise product (the core-wise Kronecker product; ranks
multiply), ``qtt_conv`` is Step 3 of Alg. 2, I = QiFFT(QFFT(F) (.) QFFT(G)),
the circular convolution of the two zero-padded arrays (Sec. 2), and
``padded_kernel`` / ``linear_part`` are the Sec. 2 padding of the kernel
samples and the extraction of the linear convolution from the circular one,
``conv_qtt_fft`` the whole of Alg. 2 with any of the three modified TT-SVDs.
"""
import numpy as np

from . import qtt as Q
from . import rsvd as RS
from . import toeplitz as T


def plain_axes(sizes):
    """Mode positions (1-based) of each axis in a plain chain holding the
    axes' bits block after block, sizes[a] bits for axis a."""
    axes, lo = [], 1
    for K in sizes:
        axes.append(list(range(lo, lo + K)))
        lo += K
    return axes


def reversed_axes(axes, d):
    """Positions of the axes' bits after ``reverse_chain``: output bit K-j,
    held by mode axes[a][j] after the transform, moves to mode d+1-axes[a][j]."""
    return [[d + 1 - m for m in reversed(pos)] for pos in axes]


def stage_operator(d, modes, p, inverse=False):
    """Operator cores O_k[left, out, in, right] (k = 1..d) of the DIF stage
    on bit p (1..K) of the axis whose bit j+1 sits on mode modes[j]: the
    butterfly on mode modes[p-1], the twiddles on modes modes[0..p-2], the
    switch passed through (bond 2) by any other mode between them, the
    identity elsewhere."""
    sgn = 1.0 if inverse else -1.0
    H = np.array([[1.0, 1.0], [1.0, -1.0]], dtype=np.complex128)
    lo, hi = modes[0], modes[p - 1]
    twid = {modes[j]: j + 1 for j in range(p - 1)}
    ops = []
    for k in range(1, d + 1):
        if k == hi:
            if p == 1:
                O = H.reshape((1, 2, 2, 1)).copy()
            else:
                # the new bit j picks the branch the lower bits see
                O = np.zeros((2, 2, 2, 1), dtype=np.complex128)
                for j in range(2):
                    O[j, j, :, 0] = H[j, :]
        elif k in twid:
            kk = twid[k]
            left = 1 if k == lo else 2
            O = np.zeros((left, 2, 2, 2), dtype=np.complex128)
            for c in range(2):
                for i in range(2):
                    t = np.exp(sgn * 2j * np.pi * i * 2.0 ** (kk - 1) / 2.0 ** p) if c else 1.0
                    O[c if left == 2 else 0, i, i, c] = t
        elif lo < k < hi:
            O = np.zeros((2, 2, 2, 2), dtype=np.complex128)
            for c in range(2):
                O[c, 0, 0, c] = O[c, 1, 1, c] = 1.0
        else:
            O = np.zeros((1, 2, 2, 1), dtype=np.complex128)
            O[0, 0, 0, 0] = O[0, 1, 1, 0] = 1.0
        ops.append(O)
    return ops


def reverse_chain(cores):
    """Mode k <- mode d+1-k (the two bonds of every core swap)."""
    return [np.transpose(c, (2, 1, 0)).copy() for c in reversed(cores)]


def _axes(axes, d):
    """The axes' mode positions, in the order the transform takes them: by
    the position of each axis' least significant bit."""
    if axes is None:
        return [list(range(1, d + 1))]
    if all(np.isscalar(a) for a in axes):
        axes = plain_axes(axes)
    return sorted((list(a) for a in axes), key=lambda a: a[0])


def qtt_fft(cores, axes=None, rmax=None, eps=0.0, inverse=False, delta=None):
    """D-dimensional DFT (inverse=True: the IDFT with its 1/N^D) of a QTT
    tensor.  axes: per axis the mode positions of its bits (LSB first), or a
    list of bit counts for a plain chain (block after block); default one
    axis of all modes; the axes are transformed in the order of their least
    significant bit's mode.  With a cap rmax, a tolerance eps or an SV drop-off
    threshold delta (Sec. 5 (1)-(3)) the input and the result of every stage
    are TT-rounded (without any the transform is exact up to rounding
    errors).  The result's chain is reversed: the axes' bits sit at
    ``reversed_axes(axes, d)``, each in natural order (a plain 2D chain comes
    out with its blocks swapped, an interleaved one with the other axis
    first)."""
    d = len(cores)
    axes = _axes(axes, d)
    assert sorted(m for a in axes for m in a) == list(range(1, d + 1))
    trunc = rmax is not None or eps > 0.0 or bool(delta)
    Y = [np.asarray(c, dtype=np.complex128) for c in cores]
    if trunc:
        Y = Q.tt_round(Y, eps, rmax, delta)
    for modes in axes:
        for p in range(len(modes), 0, -1):
            Y = T.matvec(stage_operator(d, modes, p, inverse), Y)
            if trunc:
                Y = Q.tt_round(Y, eps, rmax, delta)
    Y = reverse_chain(Y)
    if inverse:
        Y[0] = Y[0] / 2.0 ** d
    return Y


def hadamard(A, B):
    """Entrywise product of two QTT tensors on the same chain:
    Z_k[(a, a'), i, (b, b')] = A_k[a, i, b] B_k[a', i, b']."""
    out = []
    for a, b in zip(A, B):
        z = np.einsum('aib,cid->acibd', a, b)
        out.append(z.reshape((a.shape[0] * b.shape[0], 2, a.shape[2] * b.shape[2])))
    return out


def qtt_conv(F, G, axes=None, rhat=None, eps_hat=0.0, delta_hat=None):
    """Alg. 2, Step 3: QiFFT(QFFT(F) (.) QFFT(G)) with the cap rhat (or the
    tolerance eps_hat, or the drop-off threshold delta_hat) in all three
    transforms; the result is on the input chain."""
    d = len(F)
    axes = _axes(axes, d)
    Fh = qtt_fft(F, axes, rhat, eps_hat, delta=delta_hat)
    Gh = qtt_fft(G, axes, rhat, eps_hat, delta=delta_hat)
    return qtt_fft(hadamard(Fh, Gh), reversed_axes(axes, d), rhat, eps_hat, inverse=True,
                   delta=delta_hat)


def padded_kernel(taps, N, n):
    """Sec. 2 padding of the kernel: g^0_j = the kernel at grid point j of the
    N-point grid (offset j - (N-1)/2 from its centre, N odd), zero for
    N <= j < n.  taps[m + len(taps)//2] is the kernel (times the cell size)
    at offset m."""
    assert N % 2 == 1 and n >= 2 * N - 1
    c = (len(taps) - 1) // 2
    g = np.zeros(n, dtype=np.result_type(taps, np.float64))
    h = (N - 1) // 2
    for j in range(N):
        g[j] = taps[c + j - h]
    return g


def linear_part(Ic, N):
    """Sec. 2: the linear convolution I_j = I^c_{j + (N-1)/2}, j < N, per
    axis of a circular convolution of padded arrays."""
    h = (N - 1) // 2
    Ic = np.asarray(Ic)
    sl = tuple(slice(h, h + N) for _ in range(Ic.ndim))
    return Ic[sl]


def decompose(v, d, rmax, delta=None, rsvd=None):
    """Alg. 2, Step 2 with one of the modified TT-SVDs of Sec. 5: the max rank
    TT-SVD (cap rmax), the max rank TT-RSVD (rsvd = (p, omega), see
    ``rsvd.tt_rsvd``) or the SV drop-off TT-SVD (threshold delta, no cap)."""
    if delta:
        cores, _, _ = Q.tt_svd(v, d, 0.0, None, delta=delta)
    elif rsvd is not None:
        cores, _, _ = RS.tt_rsvd(v, d, rmax, rsvd[0], rsvd[1])
    else:
        cores, _, _ = Q.tt_svd(v, d, 0.0, rmax)
    return cores


def conv_qtt_fft(F0, G0, rmax, rhat, eps_hat=0.0, delta=None, rsvd=None, interleave=False):
    """Alg. 2 on padded arrays of 2^K entries per axis (a vector, or an image
    in the plain chain -- the column index' bits, then the row index' bits --
    or, with interleave, the bit-interleaved chain of ``qtt.mode_map_2d``):
    Steps 1-2 by ``decompose``, Step 3 with the cap rhat (or the tolerance
    eps_hat; with delta, the same drop-off threshold in the transforms, as
    Sec. 5 prescribes), Step 4 by Full (Alg. 3).  Returns the circular
    convolution I^c."""
    F0 = np.asarray(F0, dtype=np.complex128)
    G0 = np.asarray(G0, dtype=np.complex128)
    if F0.ndim == 1:
        d = F0.size.bit_length() - 1
        axes = [list(range(1, d + 1))]
        f, g = F0, G0
    else:
        ny, nx = F0.shape
        dx, dy = nx.bit_length() - 1, ny.bit_length() - 1
        d = dx + dy
        modes = Q.mode_map_2d(dx, dy, interleave)
        axes = [[m + 1 for m, (ax, _) in enumerate(modes) if ax == a] for a in (0, 1)]
        f = Q.image_to_qtt_vector(F0, interleave=interleave)
        g = Q.image_to_qtt_vector(G0, interleave=interleave)
    F = decompose(f, d, rmax, delta, rsvd)
    G = decompose(g, d, rmax, delta, rsvd)
    v = Q.full(qtt_conv(F, G, axes, rhat, eps_hat, delta))
    if F0.ndim == 1:
        return v
    return Q.qtt_vector_to_image(v, ny, nx, interleave=interleave)


def conv_qtt_fft_spread(F0, G0, rmax, rhat, ref, draws=3, rel=1e-7, seed=11):
    """Sensitivity of ``conv_qtt_fft`` to FP32-sized errors (a check on how
    well the capped rounding chain is conditioned, not a step of Alg. 2):
    the largest relative l2 move of the result, over ``draws`` seeded runs,
    when every core is multiplied by (1 + rel z), z complex standard normal,
    before each TT-rounding of the route (the TT-SVDs and every transform
    stage).  A GPU path computing in FP32 is compared with the FP64 route
    within a multiple of this spread."""
    rng = np.random.default_rng(seed)
    plain = Q.tt_round

    def perturbed(Y, eps, rm=None, delta=None):
        Y = [c * (1 + rel * (rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)))
             for c in Y]
        return plain(Y, eps, rm, delta)

    ref = np.asarray(ref)
    spread = 0.0
    Q.tt_round = perturbed
    try:
        for _ in range(draws):
            out = conv_qtt_fft(F0, G0, rmax, rhat)
            spread = max(spread, float(np.linalg.norm(out - ref) / np.linalg.norm(ref)))
    finally:
        Q.tt_round = plain
    return spread
