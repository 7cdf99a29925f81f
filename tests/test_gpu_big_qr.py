"""The blocked Householder QR of the large-rank rounding on its own
(qtt_debug_big_qr): the orthonormal basis that the randomised range finder
of Sec. 5's sketched TT-rounding takes from each sketch.  Checked against
what the factorisation fixes whatever its arithmetic: Q^H Q = I, Q^H A
upper triangular (A = Q R) and, with nq = n, A = Q (Q^H A) -- on ragged
shapes that span several 16-column panels and a short last panel, rank
deficient inputs (zero and repeated columns), and data scales whose squares
leave the FP32 range (the panel's rescaled norm)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _rand(rng, m, n, cplx):
    a = rng.standard_normal((m, n))
    if cplx:
        a = a + 1j * rng.standard_normal((m, n))
    return a


def _run(qlib, A, nq, cplx):
    import torch
    dt = torch.complex64 if cplx else torch.float64
    At = torch.from_numpy(A.astype(np.complex64 if cplx else np.float64)).cuda()
    Q = qlib.big_qr(At, nq).cpu().numpy().astype(np.complex128 if cplx else np.float64)
    return At.cpu().numpy().astype(np.complex128 if cplx else np.float64), Q


def _check(A, Q, cplx, rtol):
    m, n = A.shape
    nq = Q.shape[1]
    eye = Q.conj().T @ Q
    assert np.abs(eye - np.eye(nq)).max() <= rtol, np.abs(eye - np.eye(nq)).max()
    R = Q.conj().T @ A                                 # nq x n
    nrm = max(np.linalg.norm(A, 2), 1e-300)
    low = np.tril(R, -1)
    assert np.linalg.norm(low) <= rtol * nrm * np.sqrt(n)
    if nq >= min(m, n):
        assert np.linalg.norm(A - Q @ R) <= rtol * nrm * np.sqrt(n)


U32 = 2.0 ** -24


@pytest.mark.parametrize("m,n,nq,cplx", [
    (768, 384, 384, True),      # the range finder's largest regular cut (sketch 384)
    (1000, 517, 517, True),     # ragged: 33 panels, the last of 5 columns
    (300, 300, 300, True),      # square
    (1024, 64, 64, True),       # the row limit
    (97, 33, 97, True),         # full Q (nq = m > n)
    (200, 40, 7, True),         # fewer Q columns than the factorisation
    (500, 130, 130, False),     # the FP64 instantiation
])
def test_big_qr_orthonormal_and_triangular(qlib, m, n, nq, cplx):
    rng = np.random.default_rng(m + 3 * n + nq)
    A, Q = _run(qlib, _rand(rng, m, n, cplx), nq, cplx)
    tol = (60 * U32 * np.sqrt(m)) if cplx else 1e-12
    _check(A, Q, cplx, tol)


def test_big_qr_rank_deficient(qlib):
    """Zero columns, repeated columns and a rank-5 block: Householder QR
    still gives an orthonormal Q and A = Q R."""
    rng = np.random.default_rng(3)
    m, n = 640, 96
    A = _rand(rng, m, n, True)
    A[:, 10] = 0
    A[:, 20:40] = A[:, 0:1] * rng.standard_normal(20)      # multiples of one column
    A[:, 50:96] = _rand(rng, m, 5, True) @ _rand(rng, 5, 46, True)   # rank 5
    A[:, 17] = A[:, 16]
    A, Q = _run(qlib, A, n, True)
    _check(A, Q, True, 60 * U32 * np.sqrt(m))


@pytest.mark.parametrize("scale", [1e-25, 1e25])
def test_big_qr_extreme_scales(qlib, scale):
    """Entries whose squares under- or overflow FP32: the panel measures such
    columns again with the rescaled sum, so Q is the same as for the
    unscaled matrix up to rounding."""
    rng = np.random.default_rng(4)
    m, n = 300, 40
    A0 = _rand(rng, m, n, True)
    A, Q = _run(qlib, A0 * scale, n, True)
    _, Q1 = _run(qlib, A0, n, True)
    _check(A / scale, Q, True, 60 * U32 * np.sqrt(m))
    assert np.abs(Q - Q1).max() <= 1e-4


def test_big_qr_arguments(qlib):
    import torch
    A = torch.zeros((1025, 4), dtype=torch.complex64, device="cuda")
    with pytest.raises(qlib.QTTError):
        qlib.big_qr(A, 4)                       # above the row limit
    with pytest.raises(qlib.QTTError):
        qlib.big_qr(A[:10], 11)                 # nq > m
