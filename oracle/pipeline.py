"""The oracle's textbook QTT chain ("O2") and the deconvolution loss.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  float64/complex128.

conv_sinc_qtt follows Alg. 2 with the convolution step done by the QTT
Toeplitz operator (Sec. 1, [KKT13]) instead of QTT-FFT:
  step 1  reshape to QTT order (Sec. 4; 2D in the chosen bit order),
  step 2  TT-SVD with the max-rank modification (Alg. 1, Sec. 5 (1)),
  step 3  Y = round(T_x X), then for 2D Y = round(T_y Y) (one rounding per
          axis: the interleaved 2D operator T_y (x) T_x has squared ranks),
  step 4  Full (Alg. 3), back to the array order.
"""
import numpy as np

from . import qtt as Q
from . import conv as C
from . import toeplitz as T


def decompose(x, eps, rmax, interleave=True, delta=None):
    """Steps 1-2.  x: 1D vector of length 2^d or 2D image (2^dy, 2^dx).
    delta: SV drop-off rule instead of eps (Sec. 5 modification (3))."""
    x = np.asarray(x)
    if x.ndim == 1:
        v = x.astype(np.result_type(x, np.float64))
    else:
        v = Q.image_to_qtt_vector(x.astype(np.result_type(x, np.float64)), interleave)
    d = int(np.log2(v.size))
    cores, ranks, sig = Q.tt_svd(v, d, eps, rmax, delta)
    return cores, ranks, sig


def sinc_operators(shape, B, normalize=True, eps_op=1e-12, interleave=True):
    """QTT operator(s) for the sinc convolution on a 1D or 2D grid.

    shape : (n,) or (ny, nx).  B : scalar or (Bx, By).
    Returns a list of operators (each a list of cores over all QTT modes),
    applied one after the other.
    """
    if len(shape) == 1:
        taps = C.sinc_taps(shape[0], B, normalize)
        return [T.toeplitz_qtt(taps, eps_op)]
    ny, nx = shape
    Bx, By = (B, B) if np.isscalar(B) else B
    dx, dy = int(np.log2(nx)), int(np.log2(ny))
    modes = Q.mode_map_2d(dx, dy, interleave)
    ox = T.toeplitz_qtt(C.sinc_taps(nx, Bx, normalize), eps_op)
    oy = T.toeplitz_qtt(C.sinc_taps(ny, By, normalize), eps_op)
    return [T.embed_axis_operator(ox, modes, 0), T.embed_axis_operator(oy, modes, 1)]


def convolve_qtt(cores, operators, eps_round, rround=None):
    """Step 3: Y = round(O X) for each operator in turn."""
    Y = cores
    for ops in operators:
        Y = T.matvec(ops, Y)
        Y = Q.tt_round(Y, eps_round, rround)
    return Y


def to_array(cores, shape, interleave=True):
    """Step 4: Full (Alg. 3) and back to array order."""
    v = Q.full(cores)
    if len(shape) == 1:
        return v
    return Q.qtt_vector_to_image(v, shape[0], shape[1], interleave)


def conv_sinc_qtt(x, B, eps, rmax, eps_op=1e-12, eps_round=1e-12, rround=None,
                  normalize=True, interleave=True, return_parts=False):
    """decompose -> QTT Toeplitz convolution + rounding -> full."""
    x = np.asarray(x)
    cores, ranks, _ = decompose(x, eps, rmax, interleave)
    ops = sinc_operators(x.shape, B, normalize, eps_op, interleave)
    Y = convolve_qtt(cores, ops, eps_round, rround)
    out = to_array(Y, x.shape, interleave)
    if return_parts:
        return out, dict(ranks=ranks, cores=cores, y=Y, y_ranks=Q.ranks_of(Y))
    return out


def conv_dense(x, B, normalize=True):
    """O1: the plain definition (Eq. dconv) on the dense array, via FFT."""
    x = np.asarray(x)
    if x.ndim == 1:
        return C.conv_fft(x.astype(np.result_type(x, np.float64)), C.sinc_taps(x.size, B, normalize))
    ny, nx = x.shape
    Bx, By = (B, B) if np.isscalar(B) else B
    return C.conv2d_fft(x.astype(np.result_type(x, np.float64)),
                        C.sinc_taps(nx, Bx, normalize), C.sinc_taps(ny, By, normalize))


# --------------------------------------------------------------------------
# Deconvolution loss and its gradient (the differentiable use of the
# convolution step): L(F) = || full(T F) - g ||_2^2 for a QTT tensor F.
# T is the sinc Toeplitz operator; for the real even kernel T^H = T.
# Gradient convention: the one PyTorch uses for complex leaves, i.e.
# 2 dL/d conj(F_k); for real data it is the ordinary gradient.
# --------------------------------------------------------------------------
def apply_T_dense(v, shape, B, normalize=True):
    """T v on the dense array (Eq. dconv via FFT)."""
    return conv_dense(np.asarray(v).reshape(shape), B, normalize)


def deconv_loss(cores, shape, B, g, normalize=True, interleave=True):
    f = to_array(cores, shape, interleave)
    r = apply_T_dense(f, shape, B, normalize) - g
    return float(np.vdot(r, r).real)


def deconv_dense_grad(cores, shape, B, g, normalize=True, interleave=True):
    """w = 2 T^H (T f - g) on the dense array (T^H = T for the even real sinc)."""
    f = to_array(cores, shape, interleave)
    r = apply_T_dense(f, shape, B, normalize) - g
    return 2.0 * apply_T_dense(r, shape, B, normalize)


def core_grads(cores, w_qtt_vector):
    """grad_k[a, i, b] = sum over the other indices of w * conj(left partial)
    * conj(right partial): the chain rule through f = F_1 ... F_d.

    w_qtt_vector: the dense w in QTT order (length 2^d).
    """
    d = len(cores)
    grads = []
    for k in range(d):
        # left partial products of modes < k: (2^k, r_{k-1}); right: (r_k, 2^{d-k-1})
        Lp = np.ones((1, 1), dtype=cores[0].dtype) if k == 0 else _left_partial(cores[:k])
        Rp = _right_partial(cores[k + 1:]) if k < d - 1 else np.ones((1, 1), dtype=cores[0].dtype)
        nl, nr = Lp.shape[0], Rp.shape[1]
        W = w_qtt_vector.reshape((nl, 2, nr), order='F')
        gk = np.einsum('lir,la,br->aib', W, np.conj(Lp), np.conj(Rp))
        grads.append(gk)
    return grads


def _left_partial(cores):
    """(2^k, r_k) matrix of the first k cores, row index low bits first."""
    A = cores[0].reshape((2, -1), order='F')
    for c in cores[1:]:
        rp = c.shape[0]
        A = A.reshape((-1, rp), order='F') @ c.reshape((rp, -1), order='F')
    return A.reshape((-1, cores[-1].shape[2]), order='F')


def _right_partial(cores):
    """(r_k, 2^{d-k}) matrix of the cores after the cut, column index low bits first."""
    R = cores[-1].reshape((cores[-1].shape[0], 2), order='F')
    for c in reversed(cores[:-1]):
        r0, _, r1 = c.shape
        # R_new[a, i + 2 rest] = sum_b c[a, i, b] R[b, rest]
        R = np.einsum('aib,bz->aiz', c, R).reshape((r0, -1), order='F')
    return R
