"""Pins of the oracle's QTT Toeplitz operator and pipeline.  CPU only.

* the dense matrix rebuilt from the operator cores equals c(j - i) (a wrong
  borrow rule, t bit or absorbed last core fails this);
* symmetry of the even sinc kernel's operator;
* operator x vector equals the dense product (wrong index combination fails);
* the whole chain (O2) equals the plain definition (O1) when nothing is
  truncated;
* the truncated chain approximates O1 within the truncation budgets.
"""
import numpy as np
import pytest

from oracle import qtt as Q, conv as C, toeplitz as T, pipeline as P


@pytest.mark.parametrize("d,B", [(3, 2.0), (5, 6.0), (7, 20.0), (8, 16.0)])
def test_operator_dense_equals_toeplitz(d, B):
    taps = C.sinc_taps(2 ** d, B)
    ops = T.toeplitz_qtt(taps, 1e-14)
    Tq = T.operator_dense(ops)
    Td = C.toeplitz_dense(taps)
    assert np.abs(Tq - Td).max() <= 1e-13 * np.abs(Td).max()
    assert np.abs(Tq - Tq.T).max() <= 1e-13 * np.abs(Td).max()


def test_operator_generic_nonsymmetric_kernel():
    # the borrow construction must hold for any generating vector, not only even ones
    d = 6
    rng = np.random.default_rng(1)
    taps = rng.standard_normal(2 ** (d + 1) - 1)
    ops = T.toeplitz_qtt(taps, 0.0)
    assert np.abs(T.operator_dense(ops) - C.toeplitz_dense(taps)).max() <= 1e-12


def test_operator_ranks_are_twice_generating_ranks():
    d = 10
    taps = C.sinc_taps(2 ** d, 40.0)
    G, rho, _ = Q.tt_svd(T.generating_vector(taps), d + 1, 1e-10)
    ops = T.toeplitz_qtt(taps, 1e-10)
    assert [o.shape[3] for o in ops[:-1]] == [2 * r for r in rho[1:d]]


def test_matvec_equals_dense():
    d = 8
    rng = np.random.default_rng(3)
    v = rng.standard_normal(2 ** d) + 1j * rng.standard_normal(2 ** d)
    cores, _, _ = Q.tt_svd(v, d, 0.0)
    taps = C.sinc_taps(2 ** d, 9.0)
    y = T.matvec(T.toeplitz_qtt(taps, 1e-14), cores)
    assert np.linalg.norm(Q.full(y) - C.conv_direct(v, taps)) <= 1e-12 * np.linalg.norm(v)


def test_identity_embedding_2d():
    dy, dx = 3, 4
    rng = np.random.default_rng(6)
    F = rng.standard_normal((2 ** dy, 2 ** dx))
    tx, ty = C.sinc_taps(2 ** dx, 3.0), C.sinc_taps(2 ** dy, 2.0)
    for inter in (True, False):
        v = Q.image_to_qtt_vector(F, inter)
        cores, _, _ = Q.tt_svd(v, dx + dy, 0.0)
        modes = Q.mode_map_2d(dx, dy, inter)
        ox = T.embed_axis_operator(T.toeplitz_qtt(tx, 1e-14), modes, 0)
        oy = T.embed_axis_operator(T.toeplitz_qtt(ty, 1e-14), modes, 1)
        y = T.matvec(oy, T.matvec(ox, cores))
        out = Q.qtt_vector_to_image(Q.full(y), 2 ** dy, 2 ** dx, inter)
        assert np.abs(out - C.conv2d_separable(F, tx, ty)).max() <= 1e-13


@pytest.mark.parametrize("shape", [(256,), (16, 16)])
def test_pipeline_untruncated_equals_definition(shape):
    rng = np.random.default_rng(8)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    B = 8.0
    out = P.conv_sinc_qtt(x, B, 0.0, None, eps_op=1e-14, eps_round=1e-14)
    assert C.rel_l2(out, P.conv_dense(x, B)) <= 1e-12


def test_pipeline_truncated_within_budget():
    rng = np.random.default_rng(9)
    n = 2 ** 10
    t = np.arange(n) / n
    x = np.exp(-(t - 0.5) ** 2 / 0.005) + 0.1 * rng.standard_normal(n)
    eps, eps_op, eps_round = 0.05, 1e-9, 1e-9
    out = P.conv_sinc_qtt(x, 30.0, eps, None, eps_op=eps_op, eps_round=eps_round)
    cores, _, _ = Q.tt_svd(x, 10, eps)
    ref = P.conv_dense(Q.full(cores), 30.0)
    # operator and rounding errors only (the decomposition is shared)
    assert C.rel_l2(out, ref) <= 50 * (eps_op + eps_round)
