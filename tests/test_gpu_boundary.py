"""Boundary parameters of qtt_trunc through the C ABI: forced ranks (the
parity mode that takes the oracle's rank decisions, so near-threshold
singular values cannot flip a rank) and the precision selector.

* TT-SVD with fixed_ranks = the oracle's eps-ranks (Alg. 1): the same ranks
  and the oracle's reconstruction, FP64 at 1e-12 and complex64 at 1e-5;
* the rounding of the convolution with fixed_ranks = the ranks of the
  oracle's textbook rounding: the oracle's ranks exactly and its result at
  1e-5;
* QTT_PREC_FP32 on complex64 equals QTT_PREC_AUTO bit for bit.
"""
import numpy as np
import pytest

from oracle import conv as C, pipeline as P, qtt as Q
import synth

pytestmark = pytest.mark.gpu


def _line(n, seed):
    rng = synth.config_rng(0, sub=seed)
    return synth.line_1d_bumps(rng, n)[0]


def test_decompose_fixed_ranks_fp64(qlib):
    import torch
    d, eps = 12, 1e-2
    x = _line(2 ** d, 1)
    cores, ranks, _ = P.decompose(x, eps, None)
    t = qlib.qtt_decompose(torch.from_numpy(x).cuda(), eps=0.3, rmax=2, refine=True,
                           fixed_ranks=ranks)          # eps and rmax are not used
    assert t.ranks() == ranks
    got = qlib.qtt_to_full(t).cpu().numpy()
    ref = Q.full(cores)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_decompose_fixed_ranks_c64_2d(qlib):
    import torch
    n = 64
    rng = synth.config_rng(2, sub=7)
    _, clean = synth.image_2d_scene(rng, n, n, nscat=3, nrect=2, snr_db=60.0, rect_max=32)
    cores, ranks, _ = P.decompose(clean, 1e-4, None, True)
    t = qlib.qtt_decompose(torch.from_numpy(clean.astype(np.complex64)).cuda(), refine=True,
                           fixed_ranks=ranks)
    assert t.ranks() == ranks
    got = qlib.qtt_to_full(t).cpu().numpy().astype(np.complex128)
    ref = P.to_array(cores, clean.shape, True)
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


def test_rounding_fixed_ranks(qlib):
    import torch
    d, B = 12, 64.0
    rng = synth.config_rng(1, sub=9)
    x, _ = synth.line_1d_scatterers(rng, 2 ** d, nscat=8, snr_db=40.0)
    ref, parts = P.conv_sinc_qtt(x, B, 0.0, 16, eps_op=1e-7, eps_round=1e-7, return_parts=True)
    yr = parts["y_ranks"]
    f = qlib.qtt_decompose(torch.from_numpy(x.astype(np.complex64)).cuda(), eps=0.0, rmax=16,
                           refine=True)
    assert f.ranks() == parts["ranks"]
    y = qlib.qtt_conv_sinc(f, B, eps_op=1e-7, eps_round=0.5, fixed_ranks=yr)
    assert y.ranks() == yr
    got = qlib.qtt_to_full(y).cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


def test_prec_fp32_is_the_default_for_complex64(qlib):
    import torch
    x = torch.from_numpy(_line(2 ** 12, 3).astype(np.complex64)).cuda()
    a = qlib.qtt_to_full(qlib.qtt_decompose(x, rmax=16, refine=True)).cpu().numpy()
    b = qlib.qtt_to_full(qlib.qtt_decompose(x, rmax=16, refine=True,
                                            prec=qlib.QTT_PREC_FP32)).cpu().numpy()
    assert np.array_equal(a, b)
    with pytest.raises(qlib.QTTError):
        qlib.qtt_decompose(x, rmax=16, prec=qlib.QTT_PREC_FP64)
    with pytest.raises(qlib.QTTError):
        qlib.qtt_decompose(x, rmax=16, prec=qlib.QTT_PREC_BF16_REFINED)


def test_near_threshold_margin(qlib):
    """A cut whose discarded tail sits 1e-6 relative below tau (Alg. 1's
    eps-rank rule): the FP64 path decides the oracle's rank and reports a
    margin of that size; the FP32 path reports a margin at its resolution,
    and with the oracle's ranks forced it reproduces the oracle."""
    import torch
    d = 10
    x = _line(2 ** d, 4)
    _, _, sig = P.decompose(x, 0.0, None)
    s0, s1 = sig[0][0], sig[0][1]                 # the 2 x 2^(d-1) unfolding of cut 1
    eps = s1 * (1 + 1e-6) * np.sqrt(d - 1) / np.linalg.norm(x)
    cores, ranks, _ = P.decompose(x, eps, None)
    assert ranks[1] == 1 and s1 / s0 > 1e-3
    t = qlib.qtt_decompose(torch.from_numpy(x).cuda(), eps=eps, refine=True)
    m = t.margins()
    assert t.ranks() == ranks
    assert 0.0 <= m[1] < 1e-5                     # near the threshold, and reported as such
    assert np.isnan(m[0]) and np.isnan(m[d])
    got = qlib.qtt_to_full(t).cpu().numpy()
    ref = Q.full(cores)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    # FP32: the decision may go either way at this margin; forced ranks agree
    x32 = torch.from_numpy(x.astype(np.complex64)).cuda()
    t32 = qlib.qtt_decompose(x32, eps=eps, refine=True)
    assert t32.margins()[1] < 1e-3
    f32 = qlib.qtt_decompose(x32, refine=True, fixed_ranks=ranks)
    got = qlib.qtt_to_full(f32).cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
