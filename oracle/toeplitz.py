"""QTT Toeplitz operator of the sinc kernel and operator x vector contraction.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  float64/complex128.

The paper cites the QTT representation of (multilevel) Toeplitz matrices
(Sec. 1, [KKT13]) but gives no formula; this module derives it from binary
subtraction, in the oracle's own words:

  T[j, i] = c(j - i), j, i in [0, 2^d).  Put t = j - i + 2^d in [1, 2^{d+1}).
  The generating vector chat[t] = c(t - 2^d) (chat[0] = 0, never used) has
  d+1 QTT cores G_1..G_{d+1} (computed with TT-SVD, Alg. 1).  The bits of t
  follow from those of j and i by the borrow chain of the subtraction j - i:
      diff_k = j_k - i_k - b_k,  t_k = diff_k mod 2,  b_{k+1} = [diff_k < 0],
  with b_1 = 0, and t_{d+1} = 1 - b_{d+1} (adding 2^d).  So
      T[j, i] = G_1[t_1] ... G_d[t_d] G_{d+1}[t_{d+1}]
  and the operator core k, indexed by (borrow in, alpha), j_k, i_k,
  (borrow out, beta), holds G_k[alpha, t_k, beta] at the one borrow-out the
  bits determine and zero elsewhere; the last core absorbs G_{d+1}.

An operator core is a numpy 4-array O[p, j, i, q] of shape (R_{k-1}, 2, 2, R_k).
The combined operator rank index is p = b * rho + alpha.
"""
import numpy as np

from .qtt import tt_svd, mode_map_2d


def generating_vector(taps):
    """chat[t] = c(t - n) for t = 1..2n-1, chat[0] = 0 (length 2n = 2^{d+1})."""
    n = (len(taps) + 1) // 2
    chat = np.zeros(2 * n, dtype=taps.dtype)
    chat[1:] = taps            # taps[m + n - 1] = c(m)  ->  chat[m + n] = c(m)
    return chat


def toeplitz_qtt(taps, eps_op):
    """QTT operator cores (list of (R, 2, 2, R') arrays) of T[j, i] = c(j - i)."""
    n = (len(taps) + 1) // 2
    d = int(np.log2(n))
    assert 2 ** d == n
    chat = generating_vector(taps)
    G, _, _ = tt_svd(chat, d + 1, eps_op)
    ops = []
    for k in range(d):
        g = G[k]
        rho0, _, rho1 = g.shape
        nb_in = 1 if k == 0 else 2
        last = (k == d - 1)
        nq = 1 if last else 2 * rho1
        O = np.zeros((nb_in * rho0, 2, 2, nq), dtype=g.dtype)
        for b in range(nb_in):
            for j in range(2):
                for i in range(2):
                    diff = j - i - b
                    t = diff % 2
                    bout = 1 if diff < 0 else 0
                    blk = g[:, t, :]                         # rho0 x rho1
                    if last:
                        # absorb G_{d+1} at t_{d+1} = 1 - b_{d+1}
                        blk = blk @ G[d][:, 1 - bout, 0]
                        O[b * rho0:(b + 1) * rho0, j, i, 0] = blk
                    else:
                        O[b * rho0:(b + 1) * rho0, j, i,
                          bout * rho1:(bout + 1) * rho1] = blk
        ops.append(O)
    return ops


def operator_dense(ops):
    """Dense 2^d x 2^d matrix of a QTT operator (small d only).

    Row index j = sum_k j_k 2^{k-1}, column i likewise.
    """
    d = len(ops)
    n = 2 ** d
    T = np.zeros((n, n), dtype=ops[0].dtype)
    for j in range(n):
        for i in range(n):
            v = np.ones((1,), dtype=ops[0].dtype)
            for k in range(d):
                jk = (j >> k) & 1
                ik = (i >> k) & 1
                v = v @ ops[k][:, jk, ik, :]
            T[j, i] = v[0]
    return T


def identity_core(rank, dtype):
    """Pass-through operator core on a mode the operator does not act on."""
    O = np.zeros((rank, 2, 2, rank), dtype=dtype)
    for j in range(2):
        O[:, j, j, :] = np.eye(rank, dtype=dtype)
    return O


def embed_axis_operator(ops_axis, modes, axis):
    """Operator cores on all QTT modes of an image for one axis' 1D operator.

    modes : the (axis, bit) list of mode_map_2d.  Modes of the other axis get
    identity cores that carry the current rank through.
    """
    out = []
    rank = 1
    for (ax, bit) in modes:
        if ax == axis:
            O = ops_axis[bit]
            assert O.shape[0] == rank
            out.append(O)
            rank = O.shape[3]
        else:
            out.append(identity_core(rank, ops_axis[0].dtype))
    assert rank == 1
    return out


def matvec(ops, cores):
    """Operator x vector, core by core (Y = T X in QTT).

    Y_k[(p, a), j, (q, b)] = sum_i O_k[p, j, i, q] X_k[a, i, b], combined rank
    index p * r + a.  No truncation: ranks multiply.
    """
    out = []
    for O, X in zip(ops, cores):
        P, _, _, Q = O.shape
        a, _, b = X.shape
        Y = np.einsum('pjiq,aib->pajqb', O, X)
        out.append(Y.reshape((P * a, 2, Q * b)))
    return out
