"""The large-rank mode of the rounding (sketch rank above 64, complex64)
through the C ABI, for 2D images whose convolved QTT has ranks above 64
(Alg. 2 on images: the interleaved QTT of a filtered image needs ranks of a
few hundred at its middle cuts).

The oracle side is the plain definition: full(X) convolved by the dense
separable Toeplitz product of Eq. dconv (O1), with X the same seeded cores,
or the oracle's own TT-SVD (Alg. 1) of the same seeded scene.  The rounding
is an approximation, so the check is the result, not its ranks:

* exact regime: random rank-<=64 cores on 256 x 256 (every cut's rank is at
  most 256 <= the sketch rank, so the range finder spans the whole space and
  the rounding is exact up to FP32): E2 <= 1e-5 and the element-wise bound;
* approximate regime: a sparse noise-free scene on 1024 x 1024 (TT-SVD
  ranks <= 35 at eps 1e-6, so no cap decides the subspace; ranks of T_x X
  up to ~120 at eps 1e-7, below the sketch rank 384 and above the Lemma 5.1
  bound of the first cuts): decompose + convolve + Full against the
  oracle's TT-SVD + dense convolution at 1e-5, ranks above 64.
"""
import numpy as np
import pytest

from oracle import conv as C, pipeline as P, qtt as Q
import synth

pytestmark = pytest.mark.gpu


def _rand_cores(rng, d, r):
    ranks = [1] + [min(r, 2 ** k, 2 ** (d - k)) for k in range(1, d)] + [1]
    out = []
    for k in range(d):
        shp = (ranks[k], 2, ranks[k + 1])
        c = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)) / np.sqrt(4 * ranks[k])
        out.append(c)
    return out


def _dense_conv(img, B):
    ny, nx = img.shape
    return C.conv2d_separable(img, C.sinc_taps(nx, B), C.sinc_taps(ny, B))


def _check(got, ref, tol):
    e2 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    emax = np.abs(got - ref).max() / np.abs(ref).max()
    assert e2 <= tol, f"E2 {e2:.3e} > {tol:.1e}"
    assert emax <= 3 * tol, f"max-abs error {emax:.3e} > {3 * tol:.1e} of max |ref|"


@pytest.mark.parametrize("interleave", [True, False])
def test_large_rank_exact_regime(qlib, interleave):
    rng = np.random.default_rng(240 + int(interleave))
    d2 = 8
    cores = _rand_cores(rng, 2 * d2, 64)
    t = qlib.qtt_from_cores([c.astype(np.complex64) for c in cores], [d2, d2], interleave)
    B = 16.0
    y = qlib.qtt_conv_sinc(t, B, eps_op=1e-7, eps_round=1e-7, sketch=384)
    ranks = y.ranks()
    assert max(ranks) > 64
    assert all(r <= min(2 ** k, 2 ** (2 * d2 - k), 384) for k, r in enumerate(ranks))
    got = qlib.qtt_to_full(y).cpu().numpy().astype(np.complex128)
    img = Q.qtt_vector_to_image(Q.full(cores), 2 ** d2, 2 ** d2, interleave)
    _check(got, _dense_conv(img, B), 1e-5)


def test_large_rank_scene_1024(qlib):
    import torch
    n, B = 1024, 64.0
    rng = synth.config_rng(2, sub=1)
    _, clean = synth.image_2d_scene(rng, n, n, nscat=12, nrect=3, snr_db=60.0, rect_max=128)
    eps, rmax = 1e-6, 64
    cores, ranks, _ = P.decompose(clean, eps, rmax, True)
    assert max(ranks) < rmax                      # no cap: the decompositions agree
    ref = _dense_conv(P.to_array(cores, clean.shape, True), B)
    f = qlib.qtt_decompose(torch.from_numpy(clean.astype(np.complex64)).cuda(), eps=eps, rmax=rmax,
                           refine=True)
    y = qlib.qtt_conv_sinc(f, B, eps_op=1e-7, eps_round=1e-7, sketch=384)
    assert max(y.ranks()) > 64
    got = qlib.qtt_to_full(y).cpu().numpy().astype(np.complex128)
    _check(got, ref, 1e-5)


def test_large_rank_arguments(qlib):
    rng = np.random.default_rng(5)
    real = qlib.qtt_from_cores([c.real.copy() for c in _rand_cores(rng, 8, 8)], [4, 4])
    with pytest.raises(qlib.QTTError):
        qlib.qtt_conv_sinc(real, 8.0, sketch=128)          # float64: not in this mode
    cplx = qlib.qtt_from_cores([c.astype(np.complex64) for c in _rand_cores(rng, 8, 8)], [4, 4])
    with pytest.raises(qlib.QTTError):
        qlib.qtt_conv_sinc(cplx, 8.0, sketch=qlib.QTT_SKETCH_CAP_BIG + 1)   # above the cap


def test_large_rank_tensor_core_products(qlib):
    """The exact regime with the range finder's products on the tensor-core
    GEMM (qtt_debug_set_tc_gemm(1)): the same result at the accuracy its
    3xTF32 operands allow along the chain of products (each operand keeps
    ~2^-22 of its value; measured E2 8-9e-6 at three seeds, bound 2e-5),
    against ~2e-6 on the compensated CUDA-core GEMM that the library uses
    by default."""
    rng = np.random.default_rng(240)
    d2 = 8
    cores = _rand_cores(rng, 2 * d2, 64)
    t = qlib.qtt_from_cores([c.astype(np.complex64) for c in cores], [d2, d2], True)
    qlib.qtt_debug_set_tc_gemm(True)
    try:
        y = qlib.qtt_conv_sinc(t, 16.0, eps_op=1e-7, eps_round=1e-7, sketch=384)
        got = qlib.qtt_to_full(y).cpu().numpy().astype(np.complex128)
    finally:
        qlib.qtt_debug_set_tc_gemm(False)
    img = Q.qtt_vector_to_image(Q.full(cores), 2 ** d2, 2 ** d2, True)
    _check(got, _dense_conv(img, 16.0), 2e-5)
