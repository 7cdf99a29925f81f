"""QTT algebra of the oracle: reshape, TT-SVD, Full, TT-rounding.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  float64/complex128.

A QTT tensor is a Python list of numpy 3-arrays ``core[alpha, i, beta]`` of
shape ``(r_{k-1}, 2, r_k)`` with ``r_0 = r_d = 1`` (Sec. 4, TT format).  The
k-th unfolding uses the column-major convention of Sec. 4 (the first index
runs fastest), so the matrix that Alg. 1 factors at step k has row index
``alpha + r_{k-1} * i_k``; numpy's ``order='F'`` reshape is exactly the
MATLAB ``reshape`` the paper refers to.

Parity pins (tests/test_oracle_*.py): exact reconstruction at untruncated
ranks, the TT-SVD error bound of Sec. 4, analytically known QTT ranks
(exponential -> 1, sine -> 2, degree-p polynomial -> p+1), the unfolding
shapes of Lemma 5.1 and the storage counts of Table 6.3 / Table 6.5.
"""
import numpy as np


# --------------------------------------------------------------------------
# QTT index maps (Sec. 4, "QTT decomposition"): a vector v of length 2^K is
# the K-mode tensor V(i_1..i_K) = v(sum_k i_k 2^{k-1}), i_1 the least
# significant bit.  For a 2D image the paper only says matrices are reshaped
# "similarly"; the bit-interleaved (Morton) order is the one the 2D workload
# asks for, the plain order (all x bits, then all y bits) is the MATLAB one.
# --------------------------------------------------------------------------
def mode_map_2d(dx, dy, interleave=True):
    """List of (axis, bit) for QTT modes 1..dx+dy of an image F[y, x].

    axis 0 = x (the fast, column index of a row-major array), axis 1 = y.
    Interleaved: x_1, y_1, x_2, y_2, ... and the longer axis' remaining bits
    at the end.  Not interleaved: x_1..x_dx, y_1..y_dy.
    """
    modes = []
    if interleave:
        for b in range(max(dx, dy)):
            if b < dx:
                modes.append((0, b))
            if b < dy:
                modes.append((1, b))
    else:
        modes = [(0, b) for b in range(dx)] + [(1, b) for b in range(dy)]
    return modes


def image_to_qtt_vector(img, interleave=True):
    """Reorder a 2^dy x 2^dx image (row-major, F[y, x]) into the QTT vector.

    Brute-force definition: for every QTT index q, read its bits mode by mode
    and place them into x and y.
    """
    ny, nx = img.shape
    dx, dy = int(np.log2(nx)), int(np.log2(ny))
    modes = mode_map_2d(dx, dy, interleave)
    q = np.arange(nx * ny, dtype=np.int64)
    x = np.zeros_like(q)
    y = np.zeros_like(q)
    for pos, (axis, bit) in enumerate(modes):
        b = (q >> pos) & 1
        if axis == 0:
            x |= b << bit
        else:
            y |= b << bit
    return img[y, x].copy()


def qtt_vector_to_image(v, ny, nx, interleave=True):
    """Inverse of :func:`image_to_qtt_vector`."""
    dx, dy = int(np.log2(nx)), int(np.log2(ny))
    modes = mode_map_2d(dx, dy, interleave)
    q = np.arange(nx * ny, dtype=np.int64)
    x = np.zeros_like(q)
    y = np.zeros_like(q)
    for pos, (axis, bit) in enumerate(modes):
        b = (q >> pos) & 1
        if axis == 0:
            x |= b << bit
        else:
            y |= b << bit
    img = np.empty((ny, nx), dtype=v.dtype)
    img[y, x] = v
    return img


# --------------------------------------------------------------------------
# epsilon-rank (Sec. 4): the smallest r >= 1 whose discarded singular values
# have l2 norm <= tau (Eckart-Young), capped by R_max (Sec. 5, modification
# (1), "max rank TT-SVD").
# --------------------------------------------------------------------------
def eps_rank(s, tau, rmax=None):
    """Sec. 4 eps-rank: the smallest r >= 1 with sqrt(sum_{i>r} s_i^2) <= tau,
    then the cap.  tau = 0 (eps = 0) is the max rank TT-SVD of Sec. 5
    modification (1): no threshold at all, every singular value up to the cap
    is kept (exact zeros included), so the ranks follow Lemma 5.1's shapes."""
    s = np.asarray(s, dtype=np.float64)
    n = len(s)
    # tail[r] = sqrt(sum_{i >= r} s_i^2), r = 0..n
    tail2 = np.concatenate([np.cumsum((s ** 2)[::-1])[::-1], [0.0]])
    r = n
    for cand in range(1, n + 1):
        if tau > 0 and tail2[cand] <= tau * tau:
            r = cand
            break
    if rmax is not None and rmax > 0:
        r = min(r, rmax)
    return max(r, 1)


def drop_rank(s, delta, rmax=None):
    """Sec. 5 modification (3), "SV drop off": the first k (1-based) with
    sigma_{k+1} / sigma_k < delta keeps sigma_1..sigma_k; with no such drop
    every singular value is kept.  Then the cap R_max.  (Reading: the FIRST
    drop below delta, scanning from the largest singular value.)"""
    s = np.asarray(s, dtype=np.float64)
    r = len(s)
    for k in range(1, len(s)):
        if s[k - 1] > 0 and s[k] / s[k - 1] < delta:
            r = k
            break
    if rmax is not None and rmax > 0:
        r = min(r, rmax)
    return max(r, 1)


def tt_svd(v, d, eps, rmax=None, delta=None):
    """Alg. 1 (TT-SVD) with the max-rank modification (1) of Sec. 5.

    v    : vector of length 2^d in QTT order.
    eps  : relative accuracy; per-step threshold tau = eps/sqrt(d-1)*||v||
           (the reading of Alg. 1's threshold that keeps the total bound
           ||A - A~||_F <= eps ||A||_F of Sec. 4; the printed sqrt(M-1) with
           M = 2 would give eps*||A|| per step instead).
    rmax : rank cap R_max (None or <= 0: no cap).
    delta: if given (0 < delta < 1), the SV drop-off rule (``drop_rank``,
           Sec. 5 modification (3)) replaces the eps rule.
    Returns (cores, ranks, sigmas) where sigmas[k] are the singular values of
    the k-th unfolding (for tests of the error bound).
    """
    v = np.asarray(v)
    assert v.size == 2 ** d
    tau = (eps / np.sqrt(d - 1)) * np.linalg.norm(v) if d > 1 else 0.0
    cores, sigmas, ranks = [], [], [1]
    rest = v.reshape(-1, 1)
    r_prev = 1
    for k in range(1, d):
        m = 2 * r_prev
        A = rest.reshape((m, -1), order='F')          # unfolding m_k x n_k
        U, s, Vh = np.linalg.svd(A, full_matrices=False)
        r = drop_rank(s, delta, rmax) if delta else eps_rank(s, tau, rmax)
        cores.append(U[:, :r].reshape((r_prev, 2, r), order='F'))
        rest = s[:r, None] * Vh[:r, :]                 # A := Sigma V^*
        sigmas.append(s)
        ranks.append(r)
        r_prev = r
    cores.append(rest.reshape((r_prev, 2, 1), order='F'))
    ranks.append(1)
    return cores, ranks, sigmas


def full(cores):
    """Alg. 3 (Full): expand a QTT tensor to the vector of length 2^d."""
    A = cores[0].reshape((2, -1), order='F')
    for k in range(1, len(cores)):
        r_prev = cores[k].shape[0]
        A = A.reshape((-1, r_prev), order='F')
        B = cores[k].reshape((r_prev, -1), order='F')
        A = A @ B
    return A.reshape(-1, order='F')


def ranks_of(cores):
    return [1] + [c.shape[2] for c in cores]


def storage(cores):
    """Number of stored elements (the count Table 6.3 / 6.5 report)."""
    return int(sum(c.size for c in cores))


def norm(cores):
    """Frobenius norm of the QTT tensor by left-to-right Gram contraction."""
    P = np.ones((1, 1))
    for c in cores:
        # P'[b, b'] = sum_{a, a', i} conj(c[a, i, b]) P[a, a'] c[a', i, b']
        P = np.einsum('aib,ac,cid->bd', np.conj(c), P, c)
    return float(np.sqrt(abs(P[0, 0].real)))


def tt_round(cores, eps, rmax=None, delta=None):
    """TT-rounding (the QR + truncated-SVD sweep of the TT literature cited in Sec. 1).

    Right-to-left orthogonalisation by QR of each core's (r_{k-1}) x (2 r_k)
    unfolding, then a left-to-right sweep of truncated SVDs of the
    (2 r_{k-1}) x r_k unfoldings with tau = eps/sqrt(d-1)*||Y|| and the rank
    cap rmax, the same threshold rule as Alg. 1; with delta the SV drop-off
    rule (``drop_rank``, Sec. 5 modification (3)) replaces the eps rule, as
    in ``tt_svd``.
    """
    cores = [c.copy() for c in cores]
    d = len(cores)
    if d == 1:
        return cores
    for k in range(d - 1, 0, -1):
        r0, _, r1 = cores[k].shape
        C = cores[k].reshape((r0, 2 * r1), order='F')
        # C = L Q with Q having orthonormal rows: QR of C^H.
        Q, R = np.linalg.qr(C.conj().T)
        rn = Q.shape[1]
        cores[k] = Q.conj().T.reshape((rn, 2, r1), order='F')
        L = R.conj().T                                  # r0 x rn
        cores[k - 1] = np.einsum('aib,bc->aic', cores[k - 1], L)
    nrm = np.linalg.norm(cores[0])
    tau = (eps / np.sqrt(d - 1)) * nrm
    for k in range(0, d - 1):
        r0, _, r1 = cores[k].shape
        A = cores[k].reshape((2 * r0, r1), order='F')
        U, s, Vh = np.linalg.svd(A, full_matrices=False)
        r = drop_rank(s, delta, rmax) if delta else eps_rank(s, tau, rmax)
        cores[k] = U[:, :r].reshape((r0, 2, r), order='F')
        SV = s[:r, None] * Vh[:r, :]
        cores[k + 1] = np.einsum('ab,bic->aic', SV, cores[k + 1])
    return cores


def qtt_from_function_values(v, d, eps=1e-14):
    """TT-SVD at a tiny tolerance (used by the analytic-rank pins)."""
    cores, ranks, _ = tt_svd(v, d, eps)
    return cores, ranks
