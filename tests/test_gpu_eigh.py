"""The Hermitian eigen-solvers behind every truncation of Alg. 1 against
LAPACK (numpy.linalg.eigh, FP64), through the C ABI: solver 0 = FP32
tridiagonal (+ cluster back-transformation above n = 32), 1 = one-CTA
Jacobi, 2 = the relative-accuracy refinement Jacobi (three launches with
data-movement ordering above n = 32) run to convergence (at most 20 sweeps).

Checked quantities are gauge-free: eigenvalues, residual ||G u - lam u||,
orthonormality, and the projector onto the leading r-dimensional subspace
when a gap separates it.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _max(x):
    return float(np.max(x))


def _herm(rng, n, spectrum):
    X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Q, _ = np.linalg.qr(X)
    return (Q * spectrum) @ Q.conj().T


SPECTRA = {
    "uniform": lambda n, rng: rng.uniform(1.0, 2.0, n),
    "graded": lambda n, rng: np.logspace(0, -6, n),
    "cluster": lambda n, rng: np.concatenate([[50.0, 20.0, 10.0][:n],
                                              1.0 + 1e-3 * rng.standard_normal(max(n - 3, 0))]),
    "lowrank": lambda n, rng: np.concatenate([rng.uniform(1, 2, max(n // 4, 1)),
                                              np.zeros(n - max(n // 4, 1))]),
}


@pytest.mark.parametrize("solver", [0, 1, 2])
@pytest.mark.parametrize("n", [1, 2, 3, 7, 16, 33, 34, 64, 67, 100, 127, 128])
@pytest.mark.parametrize("kind", sorted(SPECTRA))
def test_small_eigh_c64(qlib, solver, n, kind):
    rng = np.random.default_rng(n)
    spec = SPECTRA[kind](n, rng)
    G = _herm(rng, n, spec)
    qlib.qtt_debug_set_eig_solver(solver)
    try:
        lam, U = qlib.qtt_small_eigh(G, qlib.QTT_C64)
    finally:
        qlib.qtt_debug_set_eig_solver(0)
    U = U.astype(np.complex128)
    ref = np.sort(np.linalg.eigvalsh(G))[::-1]
    gn = np.abs(ref).max()
    assert np.abs(lam - ref).max() <= 2e-5 * gn
    assert np.abs(U.conj().T @ U - np.eye(n)).max() <= 5e-6
    res = np.linalg.norm(G @ U - U * lam, axis=0).max()
    assert res <= 2e-5 * gn


@pytest.mark.parametrize("n", [2, 16, 64, 128])
def test_small_eigh_f64(qlib, n):
    rng = np.random.default_rng(n + 1)
    X = rng.standard_normal((n, n))
    Q, _ = np.linalg.qr(X)
    spec = np.logspace(0, -10, n)
    G = (Q * spec) @ Q.T
    lam, U = qlib.qtt_small_eigh(G, qlib.QTT_F64)
    ref = np.sort(np.linalg.eigvalsh(G))[::-1]
    assert np.abs(lam - ref).max() <= 1e-13
    assert np.abs(U.T @ U - np.eye(n)).max() <= 1e-12
    assert np.linalg.norm(G @ U - U * lam, axis=0).max() <= 1e-13


@pytest.mark.parametrize("solver", [0, 1, 2])
@pytest.mark.parametrize("n", [16, 64])
@pytest.mark.parametrize("scale", [1e-30, 1e25])
def test_small_eigh_c64_extreme_scales(qlib, solver, n, scale):
    """Gram matrices whose squared entries leave the FP32 range (traces far
    outside [2^-60, 2^60]): every solver works on a copy scaled by a power
    of two, so eigenvalues and eigenvectors keep the accuracy of the
    unscaled case."""
    rng = np.random.default_rng(n + 7)
    G = _herm(rng, n, SPECTRA["graded"](n, rng)) * scale
    qlib.qtt_debug_set_eig_solver(solver)
    try:
        lam, U = qlib.qtt_small_eigh(G, qlib.QTT_C64)
    finally:
        qlib.qtt_debug_set_eig_solver(0)
    U = U.astype(np.complex128)
    ref = np.sort(np.linalg.eigvalsh(G))[::-1]
    gn = np.abs(ref).max()
    assert np.all(np.isfinite(lam)) and np.all(np.isfinite(U))
    assert np.abs(lam - ref).max() <= 2e-5 * gn
    assert np.abs(U.conj().T @ U - np.eye(n)).max() <= 5e-6
    assert np.linalg.norm(G @ U - U * lam, axis=0).max() <= 2e-5 * gn


@pytest.mark.parametrize("scale", [1e-170, 1e170])
def test_small_eigh_f64_extreme_scales(qlib, scale):
    """FP64 Jacobi on a Gram whose squared entries leave the FP64 range."""
    rng = np.random.default_rng(9)
    n = 40
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    G = (Q * np.logspace(0, -10, n)) @ Q.T * scale
    lam, U = qlib.qtt_small_eigh(G, qlib.QTT_F64)
    # the checks on G / scale (numpy's norms would square entries near 1e170)
    ref = np.sort(np.linalg.eigvalsh(G / scale))[::-1]
    lam = lam / scale
    assert np.abs(lam - ref).max() <= 1e-13
    assert np.abs(U.T @ U - np.eye(n)).max() <= 1e-12
    assert np.linalg.norm((G / scale) @ U - U * lam, axis=0).max() <= 1e-13
