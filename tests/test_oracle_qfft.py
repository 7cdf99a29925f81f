"""Pins of the QTT-FFT / QTT-iFFT oracle and of the QTT convolution of
Alg. 2 (Sec. 4 QTT-FFT, Sec. 5 truncated transforms, Sec. 2 padding).

* untruncated, the QTT-FFT is the DFT of Sec. 2 (numpy's fft / fft2 on the
  full array, forward and inverse), for 1D chains and for the 2D chain of
  two axis blocks;
* closed forms: the DFT of the rank-1 exponential exp(2 pi i k0 j / n) is
  n delta_{k0}, reached with the cap R^_max = 1 in every stage;
* the stage operators have TT ranks <= 2 and are sqrt(2) times unitary (a
  wrong twiddle modulus or butterfly fails here), also for an axis whose
  bits are interleaved with another's;
* the interleaved 2D chain: numpy's fft2 read through the mirrored bit
  positions, and Alg. 2 on it = the circular convolution by fft2;
* Eq. tolerance: with the tolerance eps in each of the d + 1 roundings the
  result is within (d + 1) eps ||DFT(v)|| of the DFT;
* the Hadamard product is the entrywise product, with multiplied ranks;
* Alg. 2 at full ranks is the brute-force circular convolution (two loops),
  and the Sec. 2 extraction I_j = I^c_{j+(N-1)/2} is the linear convolution
  with the kernel samples of the N-point grid;
* Table 6.1 (tests/golden/table_6_1_errors.txt): with R_max = 10 and
  R^_max = 15 (the values Sec. 7 states for all three examples) the QTT-FFT
  route gives E2(I_QTT0) within 10 % of the printed value for Examples 1
  and 2 and within 20 % for Example 3 (whose value spreads 0.0155-0.0173
  over noise draws), and E2(I_xi) within 5 %; the SV drop-off column
  I_delta within 10 % for Examples 1 and 2 (Example 3's 0.1650 is not
  reproduced: this route gives 0.10); the TT-RSVD column
  I_QTTr in the printed order between I_QTT0 and I_xi and within a factor
  2 (its oversampling p is not printed).
"""
import os

import numpy as np
import pytest

from oracle import conv as C, qfft as QF, qtt as Q, toeplitz as T
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _random_qtt(rng, d, r):
    ranks = [1] + [min(r, 2 ** k, 2 ** (d - k)) for k in range(1, d)] + [1]
    return [rng.standard_normal((ranks[k], 2, ranks[k + 1]))
            + 1j * rng.standard_normal((ranks[k], 2, ranks[k + 1])) for k in range(d)]


@pytest.mark.parametrize("d", [1, 2, 3, 6, 9])
def test_fft_is_the_dft(d):
    rng = np.random.default_rng(40 + d)
    cores = _random_qtt(rng, d, 3)
    x = Q.full(cores)
    y = Q.full(QF.qtt_fft(cores))
    ref = np.fft.fft(x)
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()
    z = Q.full(QF.qtt_fft(cores, inverse=True))
    ref = np.fft.ifft(x)
    assert np.abs(z - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("dx,dy", [(1, 1), (2, 3), (4, 4), (5, 2)])
def test_fft_2d_is_fft2(dx, dy):
    rng = np.random.default_rng(7 * dx + dy)
    img = rng.standard_normal((2 ** dy, 2 ** dx)) + 1j * rng.standard_normal((2 ** dy, 2 ** dx))
    v = Q.image_to_qtt_vector(img, interleave=False)
    cores, _, _ = Q.tt_svd(v, dx + dy, 0.0)
    Y = QF.qtt_fft(cores, [dx, dy])
    # the output chain holds the row index' bits first: the transposed image
    got = Q.qtt_vector_to_image(Q.full(Y), 2 ** dx, 2 ** dy, interleave=False).T
    ref = np.fft.fft2(img)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    back = Q.full(QF.qtt_fft(Y, [dy, dx], inverse=True))
    assert np.abs(back - v).max() <= 1e-13 * np.abs(v).max()


@pytest.mark.parametrize("dx,dy", [(1, 1), (2, 3), (4, 4), (4, 2)])
def test_fft_2d_interleaved_is_fft2(dx, dy):
    rng = np.random.default_rng(70 * dx + dy)
    img = rng.standard_normal((2 ** dy, 2 ** dx)) + 1j * rng.standard_normal((2 ** dy, 2 ** dx))
    v = Q.image_to_qtt_vector(img, interleave=True)
    d = dx + dy
    cores, _, _ = Q.tt_svd(v, d, 0.0)
    modes = Q.mode_map_2d(dx, dy, True)
    axes = [[m + 1 for m, (ax, _) in enumerate(modes) if ax == a] for a in (0, 1)]
    Y = QF.qtt_fft(cores, axes)
    # bit (axis, b) of the input chain's position m ends at position d+1-m' of
    # the mirrored chain: read the output through the mirrored positions
    out = Q.full(Y)
    q = np.arange(2 ** d)
    kx = np.zeros_like(q)
    ky = np.zeros_like(q)
    for a, pos in enumerate(QF.reversed_axes(axes, d)):
        for b, m in enumerate(pos):
            bit = (q >> (m - 1)) & 1
            if a == 0:
                kx |= bit << b
            else:
                ky |= bit << b
    ref = np.fft.fft2(img)
    assert np.abs(out - ref[ky, kx]).max() <= 1e-13 * np.abs(ref).max()
    back = Q.full(QF.qtt_fft(Y, QF.reversed_axes(axes, d), inverse=True))
    assert np.abs(back - v).max() <= 1e-13 * np.abs(v).max()


@pytest.mark.parametrize("interleave", [False, True])
def test_alg2_2d_interleaved_chain(interleave):
    rng = np.random.default_rng(12)
    n = 8
    F0 = rng.standard_normal((n, n))
    G0 = rng.standard_normal((n, n))
    # rounding at eps 1e-14 keeps the exact ranks (<= 8) between the stages
    got = QF.conv_qtt_fft(F0, G0, rmax=n * n, rhat=None, eps_hat=1e-14, interleave=interleave)
    ref = np.real(np.fft.ifft2(np.fft.fft2(F0) * np.fft.fft2(G0)))
    assert np.allclose(got, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("k0", [0, 1, 37, 511, 1000])
def test_exponential_to_delta_at_rank_one(k0):
    d = 10
    n = 2 ** d
    # the rank-1 QTT of exp(2 pi i k0 j / n): core k holds exp(2 pi i k0 i_k 2^(k-1) / n)
    cores = [np.array([1.0, np.exp(2j * np.pi * k0 * 2.0 ** k / n)]).reshape((1, 2, 1))
             for k in range(d)]
    assert np.allclose(Q.full(cores), np.exp(2j * np.pi * k0 * np.arange(n) / n))
    Y = QF.qtt_fft(cores, rmax=1)
    assert Q.ranks_of(Y) == [1] * (d + 1)
    ref = np.zeros(n, dtype=complex)
    ref[k0] = n
    assert np.abs(Q.full(Y) - ref).max() <= 1e-11 * n


@pytest.mark.parametrize("d,modes", [(6, [1, 2, 3, 4, 5, 6]), (7, [3, 4, 5, 6]), (5, [1, 2]),
                                     (6, [1, 3, 5]), (7, [2, 3, 6, 7])])
def test_stage_operators(d, modes):
    for inverse in (False, True):
        for p in range(1, len(modes) + 1):
            ops = QF.stage_operator(d, modes, p, inverse)
            assert max(max(o.shape[0], o.shape[3]) for o in ops) <= 2
            M = T.operator_dense(ops)
            assert np.allclose(M.conj().T @ M, 2.0 * np.eye(2 ** d), atol=1e-12)


def test_tolerance_bound():
    rng = np.random.default_rng(3)
    d = 12
    for eps in (1e-1, 1e-2, 1e-3):
        # a smooth signal plus noise: the roundings do truncate
        t = np.arange(2 ** d) / 2 ** d
        x = np.exp(-30 * (t - 0.4) ** 2) * np.cos(90 * t) + 0.05 * rng.standard_normal(2 ** d)
        cores, _, _ = Q.tt_svd(x.astype(complex), d, 0.0, 24)
        xq = Q.full(cores)
        ref = np.fft.fft(xq)
        y = Q.full(QF.qtt_fft(cores, eps=eps))
        err = np.linalg.norm(y - ref)
        assert err <= (d + 1) * eps * np.linalg.norm(ref)


def test_hadamard():
    rng = np.random.default_rng(9)
    d = 8
    A = _random_qtt(rng, d, 3)
    B = _random_qtt(rng, d, 2)
    Z = QF.hadamard(A, B)
    assert np.allclose(Q.full(Z), Q.full(A) * Q.full(B), rtol=0, atol=1e-12 * np.abs(Q.full(Z)).max())
    ra, rb = Q.ranks_of(A), Q.ranks_of(B)
    assert Q.ranks_of(Z) == [a * b for a, b in zip(ra, rb)]


def _circ_loops(f, g):
    n = len(f)
    out = np.zeros(n, dtype=complex)
    for j in range(n):
        for i in range(n):
            out[j] += f[i] * g[(j - i) % n]
    return out


@pytest.mark.parametrize("K", [3, 4, 5])
def test_alg2_full_rank_is_circular_convolution(K):
    rng = np.random.default_rng(K)
    n = 2 ** K
    N = 2 ** (K - 1) - 1
    f0 = np.zeros(n)
    f0[:N] = rng.standard_normal(N)
    taps = C.sinc_taps(n, n / 4.0)
    g0 = QF.padded_kernel(taps, N, n)
    ic = QF.conv_qtt_fft(f0, g0, rmax=2 ** K, rhat=None)
    assert np.allclose(ic, _circ_loops(f0, g0), rtol=0, atol=1e-13)
    # Sec. 2: the linear part is Eq. dconv with the kernel on the N-grid offsets
    h, c = (N - 1) // 2, (len(taps) - 1) // 2
    tw = np.where(np.abs(np.arange(len(taps)) - c) <= h, taps, 0.0)[c - (N - 1):c + N]
    lin = C.conv_direct_loops(f0[:N], tw)
    assert np.allclose(QF.linear_part(ic, N).real, lin, rtol=0, atol=1e-13)


def test_alg2_2d_full_rank_is_circular_convolution():
    rng = np.random.default_rng(11)
    K = 3
    n = 2 ** K
    F0 = rng.standard_normal((n, n))
    G0 = rng.standard_normal((n, n))
    got = QF.conv_qtt_fft(F0, G0, rmax=n * n, rhat=None)
    ref = np.zeros((n, n))
    for y in range(n):
        for x in range(n):
            for yy in range(n):
                for xx in range(n):
                    ref[y, x] += F0[yy, xx] * G0[(y - yy) % n, (x - xx) % n]
    assert np.allclose(got, ref, rtol=0, atol=1e-12)


def _table(name):
    rows = []
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _grid_taps(taps, N):
    """Kernel samples at the offsets of the N-point grid (|m| <= (N-1)/2),
    laid out as Toeplitz taps for a length-N convolution."""
    h, c = (N - 1) // 2, (len(taps) - 1) // 2
    t = np.where(np.abs(np.arange(len(taps)) - c) <= h, taps, 0.0)
    return t[c - (N - 1):c + N]


def _example(example):
    """(noisy, kernel array, N, true convolution, noisy convolution) of a
    Sec. 7 example, the kernel sampled on the N-point grid (Sec. 2)."""
    row = [r for r in _table("table_6_1_errors.txt") if int(r[0]) == example][0]
    K = int(row[1])
    n = 2 ** K
    if example < 3:
        noisy, clean, N, B = synth.paper_example_1d(example, K, synth.config_rng(5, sub=example))
        taps = C.sinc_taps(n, B)
        tw = _grid_taps(taps, N)
        itrue = C.conv_fft(clean[:N], tw)
        ixi = C.conv_fft(noisy[:N], tw)
        g0 = QF.padded_kernel(taps, N, n)
    else:
        noisy, clean, N, B = synth.paper_example_2d(K, synth.config_rng(5, sub=example))
        taps = C.sinc_taps(n, B)
        tw = _grid_taps(taps, N)
        itrue = C.conv2d_fft(clean[:N, :N], tw, tw)
        ixi = C.conv2d_fft(noisy[:N, :N], tw, tw)
        g = QF.padded_kernel(taps, N, n)
        g0 = np.outer(g, g)
    return row, noisy, g0, N, itrue, ixi


def _e2(a, ref):
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("example", [1, 2, 3])
def test_table_6_1_through_qtt_fft(example):
    row, noisy, g0, N, itrue, ixi = _example(example)
    e_xi_p, e_q_p = float(row[2]), float(row[3])
    e_q = _e2(QF.linear_part(QF.conv_qtt_fft(noisy, g0, 10, 15), N), itrue)
    e_xi = _e2(ixi, itrue)
    assert abs(e_xi - e_xi_p) <= 0.05 * e_xi_p, e_xi
    # Example 3: E2 over noise draws spreads 0.0155-0.0173 (four draws)
    assert abs(e_q - e_q_p) <= (0.10 if example < 3 else 0.20) * e_q_p, e_q


@pytest.mark.parametrize("example", [1, 2])
def test_table_6_1_sv_dropoff(example):
    """I_delta: the SV drop-off TT-SVD with the printed delta and the same
    threshold in the QTT-FFT / QTT-iFFT roundings (Sec. 5)."""
    row, noisy, g0, N, itrue, _ = _example(example)
    e_p, delta = float(row[5]), float(row[6])
    e = _e2(QF.linear_part(QF.conv_qtt_fft(noisy, g0, None, None, delta=delta), N), itrue)
    assert abs(e - e_p) <= 0.10 * e_p, e


@pytest.mark.parametrize("example", [1, 2, 3])
def test_table_6_1_tt_rsvd(example):
    """I_QTTr: the max rank TT-RSVD (R_max = 10) in place of the TT-SVD.  The
    oversampling p is not printed; p = 5 keeps the randomized SVD on every
    level with m_k = 2 R_max > R_max + p.  The printed ordering holds,
    E2(I_QTT0) < E2(I_QTTr) < E2(I_xi), and the value is within a factor 2
    of the printed one."""
    row, noisy, g0, N, itrue, ixi = _example(example)
    e_r_p = float(row[4])
    d = int(row[1]) * (1 if example < 3 else 2)
    _, omega = synth.rsvd_omega_blocks(d, 10, 5, np.random.default_rng(2300 + example))
    e_r = _e2(QF.linear_part(QF.conv_qtt_fft(noisy, g0, 10, 15, rsvd=(5, omega)), N), itrue)
    e_q = _e2(QF.linear_part(QF.conv_qtt_fft(noisy, g0, 10, 15), N), itrue)
    assert e_q < e_r < _e2(ixi, itrue)
    assert e_r_p / 2 <= e_r <= 2 * e_r_p, e_r


def test_spread_helper_is_zero_without_perturbation_and_restores_rounding():
    """conv_qtt_fft_spread: no perturbation, no spread; a 1e-7 one moves the
    capped route by far less than its own truncation, and the rounding the
    route uses is the plain one again afterwards."""
    from oracle import qtt as Q
    rng = np.random.default_rng(2)
    K = 8
    n = 2 ** K
    f = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    g = QF.padded_kernel(C.sinc_taps(n, 16.0), 2 ** (K - 1) - 1, n)
    plain = Q.tt_round
    ref = QF.conv_qtt_fft(f, g, 6, 8)
    assert QF.conv_qtt_fft_spread(f, g, 6, 8, ref, draws=1, rel=0.0) == 0.0
    s = QF.conv_qtt_fft_spread(f, g, 6, 8, ref, draws=2)
    assert 0.0 < s < 1e-3
    assert Q.tt_round is plain
