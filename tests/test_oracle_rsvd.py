"""Pins of the randomized SVD and the max rank TT-RSVD oracle (App. A,
Algs. 4-5; Sec. 5 modification (2)).

* exact low rank: a rank-k matrix is reproduced to rounding (sigma_{k+1} = 0
  in Eq. rsvd_error), and its range finder spans exactly its column space;
* Eq. rsvd_error: ||A - A~||_2 <= (1 + 11 sqrt(k+p) sqrt(min(m, n)))
  sigma_{k+1}, plus sigma_{k+1} after truncating to k (the remark after
  the bound), on seeded matrices with decaying spectra;
* the error is far below the bound for a wide gap: with sigma_{k+1} /
  sigma_k = 1e-8 the leading k-dimensional subspace matches the SVD's;
* levels with min(m_k, n_k) <= R_max + p revert to the plain SVD: with a
  large p the TT-RSVD is the max rank TT-SVD;
* a vector whose QTT ranks are <= R_max is reproduced to rounding.
"""
import numpy as np
import pytest

from oracle import qtt as Q, rsvd as RS
import synth


def _spectrum_matrix(rng, m, n, s, dtype=np.float64):
    X = rng.standard_normal((m, m))
    Y = rng.standard_normal((n, n))
    if dtype == np.complex128:
        X = X + 1j * rng.standard_normal((m, m))
        Y = Y + 1j * rng.standard_normal((n, n))
    U, _ = np.linalg.qr(X)
    V, _ = np.linalg.qr(Y)
    k = len(s)
    return (U[:, :k] * s) @ V[:, :k].conj().T


@pytest.mark.parametrize("dtype", [np.float64, np.complex128])
def test_exact_low_rank(dtype):
    rng = np.random.default_rng(11)
    m, n, k, p = 60, 300, 7, 5
    A = _spectrum_matrix(rng, m, n, np.linspace(3.0, 1.0, k), dtype)
    Om = rng.standard_normal((n, k + p))
    U, s, Vh = RS.rsvd(A, Om, k)
    assert np.linalg.norm(A - (U * s) @ Vh) <= 1e-12 * np.linalg.norm(A)
    Qr = RS.range_finder(A, Om)
    assert np.linalg.norm(A - Qr @ (Qr.conj().T @ A)) <= 1e-12 * np.linalg.norm(A)
    np.testing.assert_allclose(s, np.linalg.svd(A, compute_uv=False)[:k], rtol=1e-12)


@pytest.mark.parametrize("seed", range(6))
def test_error_bound(seed):
    rng = np.random.default_rng(100 + seed)
    m, n, k, p = 80, 400, 10, 6
    s = np.exp(-0.15 * np.arange(m))
    A = _spectrum_matrix(rng, m, n, s)
    Om = rng.standard_normal((n, k + p))
    U, sk, Vh = RS.rsvd(A, Om, k)
    err = np.linalg.norm(A - (U * sk) @ Vh, 2)
    bound = (1 + 11 * np.sqrt(k + p) * np.sqrt(min(m, n))) * s[k] + s[k]
    assert err <= bound
    # the optimum is sigma_{k+1}; a plain range finder is within a small factor
    assert err >= s[k] * (1 - 1e-12)


def test_wide_gap_recovers_the_svd_subspace():
    rng = np.random.default_rng(7)
    m, n, k, p = 50, 500, 6, 4
    s = np.concatenate([np.linspace(2.0, 1.0, k), 1e-8 * np.linspace(1.0, 0.5, m - k)])
    A = _spectrum_matrix(rng, m, n, s)
    U, _, _ = RS.rsvd(A, rng.standard_normal((n, k + p)), k)
    Us = np.linalg.svd(A)[0][:, :k]
    assert np.linalg.norm(U @ U.conj().T - Us @ Us.conj().T, 2) <= 1e-6


def test_fallback_is_max_rank_tt_svd():
    rng = np.random.default_rng(3)
    d, rmax, p = 10, 8, 600          # every min(m_k, n_k) <= R_max + p
    x = rng.standard_normal(2 ** d)
    _, omega = synth.rsvd_omega_blocks(d, rmax, p, rng)
    cores, ranks, used = RS.tt_rsvd(x, d, rmax, p, omega)
    assert not any(used)
    ref, rref, _ = Q.tt_svd(x, d, 0.0, rmax)
    assert ranks == rref
    np.testing.assert_allclose(Q.full(cores), Q.full(ref), rtol=0, atol=1e-12 * np.linalg.norm(x))


@pytest.mark.parametrize("dtype", [np.float64, np.complex128])
def test_low_qtt_rank_vector_is_reproduced(dtype):
    rng = np.random.default_rng(5)
    d, r, rmax, p = 12, 3, 8, 4      # m_k = 2 R_max = 16 > R_max + p
    ranks = [1] + [min(r, 2 ** k, 2 ** (d - k)) for k in range(1, d)] + [1]
    cores = []
    for k in range(d):
        c = rng.standard_normal((ranks[k], 2, ranks[k + 1]))
        if dtype == np.complex128:
            c = c + 1j * rng.standard_normal(c.shape)
        cores.append(c)
    x = Q.full(cores)
    _, omega = synth.rsvd_omega_blocks(d, rmax, p, rng)
    got, granks, used = RS.tt_rsvd(x, d, rmax, p, omega)
    assert any(used)
    assert np.linalg.norm(Q.full(got) - x) <= 1e-11 * np.linalg.norm(x)


def test_noisy_line_error_near_tt_svd():
    """Context for the GPU mode: on a noisy line the TT-RSVD error stays
    within a small factor of the max rank TT-SVD's (the optimum per level)."""
    rng = synth.config_rng(1)
    d, rmax, p = 14, 16, 8
    x, _ = synth.line_1d_scatterers(rng, 2 ** d, nscat=30, snr_db=20.0)
    _, omega = synth.rsvd_omega_blocks(d, rmax, p, np.random.default_rng(9))
    got, ranks, used = RS.tt_rsvd(x, d, rmax, p, omega)
    ref, rref, _ = Q.tt_svd(x, d, 0.0, rmax)
    assert any(used) and ranks == rref
    e_r = np.linalg.norm(Q.full(got) - x)
    e_s = np.linalg.norm(Q.full(ref) - x)
    assert e_r <= 1.5 * e_s


def test_fallback_boundary_is_inclusive():
    """Sec. 5: a level reverts to the SVD when min(m_k, n_k) <= R_max + p,
    equality included.  d = 10, R_max = p = 8: the levels with m_k = 16 and
    n_k >= 16 sit exactly on the boundary and revert; level k = 7 with
    m_k = 16 and n_k = 8 reverts too; nothing here exceeds R_max + p."""
    rng = np.random.default_rng(21)
    d, rmax, p = 10, 8, 8
    x = rng.standard_normal(2 ** d)
    _, omega = synth.rsvd_omega_blocks(d, rmax, p, rng)
    _, ranks, used = RS.tt_rsvd(x, d, rmax, p, omega)
    assert ranks[4] == 8 and 2 * ranks[4] == rmax + p
    assert not any(used)
    # one less oversampling puts the m_k = 16 levels with n_k >= 16 above it
    _, omega = synth.rsvd_omega_blocks(d, rmax, p - 1, rng)
    _, _, used = RS.tt_rsvd(x, d, rmax, p - 1, omega)
    assert used[3:6] == [True, True, True] and not any(used[:3])
