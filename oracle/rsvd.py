"""Randomized SVD and the max rank TT-RSVD (test infrastructure: the oracle).

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs use this module;
the library never does.

* ``range_finder``: App. A, Alg. 4 -- Y = A Omega, then Q from the QR
  factorisation of Y (orthonormal columns approximating the range of A).
* ``rsvd``: App. A, Alg. 5 -- B = Q^* A, B = U~ Sigma V^*, U = Q U~,
  optionally truncated to the leading k triplets.
* ``tt_rsvd``: Sec. 5 modification (2), the max rank TT-RSVD -- Alg. 1 with
  the SVD of every unfolding A^{k} (m_k x n_k) replaced by ``rsvd`` with
  k = R_max and oversampling p, each level keeping min(R_max, ...) triplets
  (no threshold: the cap alone, as for the max rank TT-SVD); a level with
  min(m_k, n_k) <= R_max + p reverts to the plain SVD (the max rank TT-SVD).

The Gaussian test matrices are the random numbers the method draws, so they
are inputs here: ``omega(k, n, l)`` returns the n x l matrix of level k.
The unfoldings follow ``qtt.tt_svd`` (column-major reshapes, mode 1 = the
least significant bit).
"""
import numpy as np


def range_finder(A, Omega):
    """App. A, Alg. 4: Y = A Omega; Q R = Y (reduced QR)."""
    Y = A @ Omega
    Q, _ = np.linalg.qr(Y)
    return Q


def rsvd(A, Omega, k=None):
    """App. A, Alg. 5 on the range found by Alg. 4; returns (U, s, Vh), the
    leading k triplets when k is given."""
    Q = range_finder(A, Omega)
    B = Q.conj().T @ A
    Ut, s, Vh = np.linalg.svd(B, full_matrices=False)
    U = Q @ Ut
    if k is not None:
        U, s, Vh = U[:, :k], s[:k], Vh[:k]
    return U, s, Vh


def tt_rsvd(v, d, rmax, p, omega):
    """Sec. 5 modification (2), max rank TT-RSVD of a vector of length 2^d in
    QTT order.  Returns (cores, ranks, used) with used[k-1] True where level
    k took the randomized SVD."""
    v = np.asarray(v)
    assert v.size == 2 ** d and rmax >= 1 and p >= 0
    cores, ranks, used = [], [1], []
    rest = v.reshape(-1, 1)
    r_prev = 1
    for k in range(1, d):
        m = 2 * r_prev
        A = rest.reshape((m, -1), order='F')          # unfolding m_k x n_k
        n = A.shape[1]
        if min(m, n) <= rmax + p:
            U, s, Vh = np.linalg.svd(A, full_matrices=False)
            used.append(False)
        else:
            U, s, Vh = rsvd(A, omega(k, n, rmax + p))
            used.append(True)
        r = max(1, min(rmax, len(s)))
        cores.append(U[:, :r].reshape((r_prev, 2, r), order='F'))
        rest = s[:r, None] * Vh[:r, :]                 # A := Sigma V^*
        ranks.append(r)
        r_prev = r
    cores.append(rest.reshape((r_prev, 2, 1), order='F'))
    ranks.append(1)
    return cores, ranks, used
