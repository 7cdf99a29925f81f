"""The TF32-refined precision mode of the complex64 TT-SVD (qtt_prec
QTT_PREC_TF32_REFINED) through the C ABI against the FP64 oracle (Alg. 1).

In this mode the first Gram pass of every unfolding with at least 32 rows
runs on the tensor cores (TF32 operands); the second pass -- projection on
the first pass's eigenvectors, FP32 Gram, relative-accuracy Jacobi, rank
decision -- is the FP32 path's.  The bar is the FP32 path's: the oracle's
ranks exactly and E2 <= 1e-5, with an element-wise bound beside it.
"""
import ctypes

import numpy as np
import pytest

from oracle import conv as C, pipeline as P, qtt as Q
import synth

pytestmark = pytest.mark.gpu
TOL32 = 1e-5


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _tc_launches(qlib, fn):
    """Run fn with per-kernel profiling on; launches of the tensor-core Gram."""
    L = qlib.lib()
    L.qtt_profile_enable.argtypes = [ctypes.c_int]
    L.qtt_profile_read.restype = ctypes.c_int
    L.qtt_profile_read.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_int), ctypes.c_int]
    L.qtt_profile_reset()
    L.qtt_profile_enable(1)
    try:
        out = fn()
    finally:
        L.qtt_profile_enable(0)
    cap, stride = 64, 64
    names = ctypes.create_string_buffer(cap * stride)
    ms = (ctypes.c_double * cap)()
    cnt = (ctypes.c_int * cap)()
    nk = L.qtt_profile_read(names, stride, ms, cnt, cap)
    n = 0
    for i in range(nk):
        nm = names.raw[i * stride:(i + 1) * stride].split(b"\0")[0].decode()
        if nm.startswith("tc_gram"):
            n += cnt[i]
    L.qtt_profile_reset()
    return out, n


def _check(got, ref, tol):
    assert C.rel_l2(got, ref) <= tol
    assert np.abs(got - ref).max() <= 3 * tol * np.abs(ref).max()


@pytest.mark.parametrize("d,rmax,eps", [(14, 32, 0.0), (16, 64, 0.0), (16, 64, 1e-3)])
def test_tf32_refined_line(qlib, d, rmax, eps):
    rng = synth.config_rng(1, sub=d)
    x, _ = synth.line_1d_scatterers(rng, 2 ** d, nscat=30, snr_db=20.0)
    x = x.astype(np.complex64)
    t, ntc = _tc_launches(qlib, lambda: qlib.qtt_decompose(
        _dev(x), eps=eps, rmax=rmax, refine=True, prec=qlib.QTT_PREC_TF32_REFINED))
    assert ntc > 0                                # the tensor-core pass ran
    cores, oranks, _ = Q.tt_svd(x.astype(np.complex128), d, eps, rmax)
    assert t.ranks() == oranks
    _check(qlib.qtt_to_full(t).cpu().numpy().astype(np.complex128), Q.full(cores), TOL32)


def test_tf32_refined_image(qlib):
    n = 256
    rng = synth.config_rng(2, sub=5)
    x, _ = synth.image_2d_scene(rng, n, n, nscat=40, nrect=3, snr_db=10.0)
    x = x.astype(np.complex64)
    t, ntc = _tc_launches(qlib, lambda: qlib.qtt_decompose(
        _dev(x), eps=3e-2, rmax=64, refine=True, interleave=True,
        prec=qlib.QTT_PREC_TF32_REFINED))
    assert ntc > 0
    cores, oranks, _ = P.decompose(x.astype(np.complex128), 3e-2, 64, interleave=True)
    assert t.ranks() == oranks
    got = qlib.qtt_to_full(t).cpu().numpy().astype(np.complex128)
    _check(got, Q.qtt_vector_to_image(Q.full(cores), n, n, True), TOL32)


def test_tf32_refined_line_2p20(qlib):
    """The full 2^20-sample line of the benchmark's line configuration."""
    rng = synth.config_rng(1)
    x, _ = synth.line_1d_scatterers(rng, 2 ** 20, nscat=50, nbumps=3, snr_db=20.0)
    x = x.astype(np.complex64)
    t = qlib.qtt_decompose(_dev(x), eps=0.0, rmax=64, refine=True,
                           prec=qlib.QTT_PREC_TF32_REFINED)
    cores, oranks, _ = Q.tt_svd(x.astype(np.complex128), 20, 0.0, 64)
    assert t.ranks() == oranks
    _check(qlib.qtt_to_full(t).cpu().numpy().astype(np.complex128), Q.full(cores), TOL32)


def test_tf32_refined_unsupported_calls(qlib):
    x = _dev(synth.line_1d_bumps(synth.config_rng(0, sub=1), 2 ** 10)[0])
    with pytest.raises(qlib.QTTError):             # FP64 data
        qlib.qtt_decompose(x, rmax=8, prec=qlib.QTT_PREC_TF32_REFINED)
    f = qlib.qtt_decompose(x.to(dtype=__import__("torch").complex64), rmax=8, refine=True)
    with pytest.raises(qlib.QTTError):             # the rounding has no tensor-core mode
        qlib.qtt_conv_sinc(f, 32.0, prec=qlib.QTT_PREC_TF32_REFINED)
