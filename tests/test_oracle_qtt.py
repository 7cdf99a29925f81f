"""Pins of the oracle's QTT algebra (Sec. 4, Alg. 1, Alg. 3, Lemma 5.1,
Table 6.3 / 6.5, TT-rounding).  CPU only.

What pins what:
* exact reconstruction at untruncated ranks and brute-force evaluation of the
  TT product -> TT-SVD and Full (a wrong reshape order or dropped core fails);
* the error bound ||A - A~|| <= eps ||A|| and the per-step Eckart-Young
  bound sum(dropped sigma^2) <= tau^2 -> the threshold rule;
* analytic QTT ranks (exponential 1, sine/cosine 2, degree-p polynomial p+1)
  -> the eps-rank definition;
* the storage counts of Table 6.3 (golden file) -> the max-rank cap;
* Lemma 5.1 unfolding shapes;
* Morton order exhaustive bijection.
"""
import os

import numpy as np
import pytest

from oracle import qtt as Q

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _brute_eval(cores, idx):
    d = len(cores)
    v = np.ones((1,), dtype=cores[0].dtype)
    for k in range(d):
        v = v @ cores[k][:, (idx >> k) & 1, :]
    return v[0]


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("d", [4, 7, 10])
def test_exact_reconstruction(d, cplx):
    rng = np.random.default_rng(d)
    v = rng.standard_normal(2 ** d)
    if cplx:
        v = v + 1j * rng.standard_normal(2 ** d)
    cores, ranks, _ = Q.tt_svd(v, d, 0.0)
    assert ranks == [1] + [min(2 ** k, 2 ** (d - k)) for k in range(1, d)] + [1]
    assert np.linalg.norm(Q.full(cores) - v) <= 1e-13 * np.linalg.norm(v)
    for idx in rng.choice(2 ** d, 20):
        assert abs(_brute_eval(cores, int(idx)) - v[idx]) <= 1e-12 * np.abs(v).max()


def test_unfolding_is_column_major():
    # Sec. 4: alpha = i_1 + 2 i_2 + ... ; first unfolding is 2 x 2^{d-1} with row = bit 1
    d = 5
    v = np.arange(2 ** d, dtype=float)
    A = v.reshape((2, -1), order='F')
    assert np.all(A[0] == v[0::2]) and np.all(A[1] == v[1::2])


@pytest.mark.parametrize("eps", [1e-1, 3e-2, 1e-3])
def test_error_bound_and_eckart_young(eps):
    rng = np.random.default_rng(11)
    d = 12
    x = np.linspace(0, 1, 2 ** d)
    v = np.exp(-(x - 0.4) ** 2 / 0.01) + 0.05 * rng.standard_normal(2 ** d)
    cores, ranks, sig = Q.tt_svd(v, d, eps)
    nv = np.linalg.norm(v)
    err = np.linalg.norm(Q.full(cores) - v)
    assert err <= eps * nv * (1 + 1e-12)
    tau = eps / np.sqrt(d - 1) * nv
    for k in range(1, d):
        s = sig[k - 1]
        assert np.sum(s[ranks[k]:] ** 2) <= tau ** 2 * (1 + 1e-12)
        if ranks[k] > 1:                     # minimality: dropping one more would exceed tau
            assert np.sum(s[ranks[k] - 1:] ** 2) > tau ** 2


def test_lemma_5_1_shapes():
    rng = np.random.default_rng(2)
    K, R = 11, 6
    v = rng.standard_normal(2 ** K)
    cores, ranks, sig = Q.tt_svd(v, K, 0.0, R)
    for k in range(1, K):
        m_k, n_k = 2 * ranks[k - 1], 2 ** (K - k)
        assert m_k <= 2 * R
        assert len(sig[k - 1]) == min(m_k, n_k)
        assert cores[k - 1].shape == (ranks[k - 1], 2, ranks[k])


def test_analytic_qtt_ranks():
    d = 14
    x = np.arange(2 ** d) / 2 ** d
    _, r, _ = Q.tt_svd(np.exp(-3.7 * x), d, 1e-12)
    assert max(r) == 1
    _, r, _ = Q.tt_svd(np.sin(13.0 * x + 0.3), d, 1e-12)
    assert max(r) == 2
    _, r, _ = Q.tt_svd(np.exp(2j * np.pi * 5 * x), d, 1e-12)
    assert max(r) == 1
    for p in (1, 2, 3, 4):
        poly = np.polyval(np.arange(1, p + 2, dtype=float), x)
        _, r, _ = Q.tt_svd(poly, d, 1e-12)
        assert max(r) == p + 1


def _golden_storage():
    rows = []
    with open(os.path.join(GOLD, "table_6_3_storage.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append(tuple(int(t) for t in line.split()))
    return rows


@pytest.mark.parametrize("K", [16, 20])
def test_table_6_3_storage(K):
    # noise has full TT ranks, so max-rank TT-SVD with R_max = 10 hits the cap profile
    gold = {k: (full, q) for k, full, q in _golden_storage()}
    rng = np.random.default_rng(K)
    v = rng.standard_normal(2 ** K)
    cores, ranks, _ = Q.tt_svd(v, K, 0.0, 10)
    assert v.size == gold[K][0]
    assert Q.storage(cores) == gold[K][1]
    assert ranks == [1] + [min(2 ** k, 2 ** (K - k), 10) for k in range(1, K)] + [1]


def test_storage_closed_form_all_rows():
    for K, full, q in _golden_storage():
        ranks = [1] + [min(2 ** k, 2 ** (K - k), 10) for k in range(1, K)] + [1]
        assert sum(ranks[k] * 2 * ranks[k + 1] for k in range(K)) == q
        assert 2 ** K == full


@pytest.mark.parametrize("dy,dx", [(1, 1), (3, 3), (2, 5), (5, 2), (5, 5)])
@pytest.mark.parametrize("interleave", [True, False])
def test_morton_bijection(dy, dx, interleave):
    ny, nx = 2 ** dy, 2 ** dx
    img = np.arange(ny * nx).reshape(ny, nx)
    v = Q.image_to_qtt_vector(img, interleave)
    assert sorted(v.tolist()) == list(range(ny * nx))           # bijection
    assert np.array_equal(Q.qtt_vector_to_image(v, ny, nx, interleave), img)
    modes = Q.mode_map_2d(dx, dy, interleave)
    for q in range(ny * nx):                                    # bit placement
        x = sum(((q >> p) & 1) << b for p, (a, b) in enumerate(modes) if a == 0)
        y = sum(((q >> p) & 1) << b for p, (a, b) in enumerate(modes) if a == 1)
        assert v[q] == img[y, x]
    if interleave and dx == dy and dx >= 2:
        assert [m for m in modes[:4]] == [(0, 0), (1, 0), (0, 1), (1, 1)]
    if not interleave:
        assert np.array_equal(v, img.reshape(-1))                # x bits first = row-major order


def test_eps_rank_definition():
    s = np.array([4.0, 2.0, 1.0, 0.5, 0.25])
    assert Q.eps_rank(s, 0.0) == 5
    assert Q.eps_rank(s, 0.25) == 4
    assert Q.eps_rank(s, np.sqrt(0.5 ** 2 + 0.25 ** 2)) == 3
    assert Q.eps_rank(s, 100.0) == 1
    assert Q.eps_rank(s, 0.0, rmax=2) == 2
    # eps = 0 is the cap-only TT-SVD: exact zeros are kept up to the cap
    assert Q.eps_rank(np.array([3.0, 0.0, 0.0]), 0.0) == 3
    assert Q.eps_rank(np.array([3.0, 0.0, 0.0]), 1e-300) == 1


def test_round_exact_and_bounded():
    rng = np.random.default_rng(9)
    d = 10
    # a TT with redundant ranks: sum of two identical TTs
    v = np.cos(7 * np.arange(2 ** d) / 2 ** d) + 0.01 * rng.standard_normal(2 ** d)
    cores, _, _ = Q.tt_svd(v, d, 0.0)
    # pad ranks by block-diagonal doubling (exact sum v + v)
    dbl = []
    for k, c in enumerate(cores):
        a, _, b = c.shape
        if k == 0:
            dbl.append(np.concatenate([c, c], axis=2))
        elif k == d - 1:
            dbl.append(np.concatenate([c, c], axis=0))
        else:
            z = np.zeros((2 * a, 2, 2 * b))
            z[:a, :, :b] = c
            z[a:, :, b:] = c
            dbl.append(z)
    r0 = Q.tt_round(dbl, 1e-14)
    assert np.linalg.norm(Q.full(r0) - 2 * v) <= 1e-12 * np.linalg.norm(2 * v)
    assert max(Q.ranks_of(r0)) <= max(Q.ranks_of(cores))
    for eps in (1e-2, 1e-1):
        r1 = Q.tt_round(dbl, eps)
        assert np.linalg.norm(Q.full(r1) - 2 * v) <= eps * np.linalg.norm(2 * v) * (1 + 1e-10)
        r2 = Q.tt_round(r1, eps)                                  # rounding again: small change
        assert np.linalg.norm(Q.full(r2) - Q.full(r1)) <= eps * np.linalg.norm(2 * v)


def test_norm_matches_full():
    rng = np.random.default_rng(4)
    v = rng.standard_normal(2 ** 9) + 1j * rng.standard_normal(2 ** 9)
    cores, _, _ = Q.tt_svd(v, 9, 0.0)
    assert abs(Q.norm(cores) - np.linalg.norm(v)) <= 1e-12 * np.linalg.norm(v)


def test_drop_rank_rule():
    # Sec. 5 modification (3): the first relative drop below delta
    s = np.array([10.0, 9.0, 8.0, 0.1, 0.09, 0.001])
    assert Q.drop_rank(s, 0.5) == 3
    assert Q.drop_rank(s, 0.05) == 3          # 0.1 / 8 is the first ratio below 0.05
    assert Q.drop_rank(s, 0.012) == 5         # 0.1 / 8 = 0.0125 passes, 0.001 / 0.09 does not
    assert Q.drop_rank(s, 0.01) == 6          # no ratio below 0.01: keep all
    assert Q.drop_rank(s, 0.5, rmax=2) == 2
    assert Q.drop_rank(np.array([1.0, 0.0]), 0.5) == 1


def test_drop_rule_recovers_exact_qtt_ranks():
    # a sum of two exponentials has QTT rank 2 at every cut; with a small
    # perturbation the singular values drop by many orders after the 2nd
    rng = np.random.default_rng(9)
    d = 10
    i = np.arange(2 ** d)
    v = np.exp(-i / 300.0) + 0.5 * np.exp(-i / 37.0) + 1e-9 * rng.standard_normal(2 ** d)
    cores, ranks, sig = Q.tt_svd(v, d, 0.0, None, delta=1e-3)
    assert ranks[1:-1] == [2] * (d - 1)
    assert np.linalg.norm(Q.full(cores) - v) <= 1e-6 * np.linalg.norm(v)
