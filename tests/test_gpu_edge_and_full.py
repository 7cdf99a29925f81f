"""Edge cases of the C ABI path and parity at the benchmark's full sizes.

* full size: the 2^20-sample complex line of the benchmark, and sampled
  lines of the 256-line batch, against the FP64 oracle (1e-5);
* degenerate inputs: all-zero and constant signals, the smallest grids,
  rank cap 1, widely scaled data;
* argument errors come back as status codes, never as device faults.
"""
import ctypes

import numpy as np
import pytest

from oracle import qtt as Q, conv as C, pipeline as P
import synth

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _pipeline(q, x, B, eps, rmax, eps_op, eps_round, refine=True):
    f = q.qtt_decompose(_dev(x), eps=eps, rmax=rmax, refine=refine)
    y = q.qtt_conv_sinc(f, B, eps_op=eps_op, eps_round=eps_round)
    return f, y, q.qtt_to_full(y).cpu().numpy()


# ------------------------------------------------------------- full sizes
def test_line_2p20_full_size_matches_oracle(qlib):
    rng = synth.config_rng(1)
    x, _ = synth.line_1d_scatterers(rng, 2 ** 20, nscat=50, nbumps=3, snr_db=20.0)
    x = x.astype(np.complex64)
    _, _, out = _pipeline(qlib, x, 1024.0, 0.0, 64, 1e-7, 1e-7)
    ref = P.conv_sinc_qtt(x.astype(np.complex128), 1024.0, 0.0, 64, eps_op=1e-7, eps_round=1e-7)
    assert C.rel_l2(out.astype(np.complex128), ref) <= 1e-5


def test_batch_256_lines_sampled_match_oracle(qlib):
    import torch
    q = qlib
    lines = synth.batch_lines(synth.config_rng(3), nlines=256, dmin=14, dmax=18, snr_db=15.0,
                              bmin=128.0, bmax=1024.0)
    xs = [_dev(ln["x"].astype(np.complex64)) for ln in lines]
    ys = q.qtt_batch_conv_sinc(xs, [ln["B"] for ln in lines], [ln["rmax"] for ln in lines])
    torch.cuda.synchronize()
    order = sorted(range(len(lines)), key=lambda i: lines[i]["d"])
    for i in (order[0], order[1], order[-1]):
        ln = lines[i]
        ref = P.conv_sinc_qtt(ln["x"].astype(np.complex128), ln["B"], 0.0, ln["rmax"],
                              eps_op=1e-7, eps_round=1e-7)
        assert C.rel_l2(ys[i].cpu().numpy().astype(np.complex128), ref) <= 1e-5


# ------------------------------------------------------------- degenerate data
@pytest.mark.parametrize("dtype", [np.float64, np.complex64])
def test_zero_signal(qlib, dtype):
    # eps = 0 is the cap-only TT-SVD: Lemma 5.1 ranks even for exact zeros;
    # the rounding (eps > 0) then drops everything to rank 1
    x = np.zeros(2 ** 10, dtype=dtype)
    f, y, out = _pipeline(qlib, x, 40.0, 0.0, 16, 1e-7, 1e-7)
    _, ranks, _ = P.decompose(np.zeros(x.size), 0.0, 16)
    assert f.ranks() == ranks == [1, 2, 4, 8, 16, 16, 16, 8, 4, 2, 1]
    assert y.ranks() == [1] * 11
    assert np.all(out == 0)


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-12), (np.complex64, 1e-5)])
def test_constant_signal_is_rank_one(qlib, dtype, tol):
    x = np.full(2 ** 12, 0.7 - (0.2j if dtype == np.complex64 else 0.0), dtype=dtype)
    f = qlib.qtt_decompose(_dev(x), eps=1e-6, rmax=0, refine=True)
    assert f.ranks() == [1] * 13
    assert C.rel_l2(qlib.qtt_to_full(f).cpu().numpy(), x) <= tol


@pytest.mark.parametrize("shape", [(4,), (2, 2), (2, 8)])
def test_smallest_grids(qlib, shape):
    rng = np.random.default_rng(3)
    x = rng.standard_normal(shape)
    _, _, out = _pipeline(qlib, x, 2.0, 0.0, 0, 1e-12, 1e-12)
    ref = P.conv_sinc_qtt(x, 2.0, 0.0, None, eps_op=1e-12, eps_round=1e-12)
    assert C.rel_l2(out, ref) <= 1e-11
    assert C.rel_l2(ref, P.conv_dense(x, 2.0)) <= 1e-11


def test_rank_cap_one(qlib):
    rng = np.random.default_rng(4)
    x = rng.standard_normal(2 ** 10)
    f = qlib.qtt_decompose(_dev(x), eps=0.0, rmax=1, refine=True)
    assert f.ranks() == [1] * 11
    cores, ranks, _ = P.decompose(x, 0.0, 1)
    assert C.rel_l2(qlib.qtt_to_full(f).cpu().numpy(), Q.full(cores)) <= 1e-12


def test_rank_cap_above_capacity_is_clamped(qlib):
    rng = np.random.default_rng(5)
    x = rng.standard_normal(2 ** 16).astype(np.complex64)
    f = qlib.qtt_decompose(_dev(x), eps=0.0, rmax=500, refine=True)
    assert max(f.ranks()) <= qlib.QTT_RANK_CAP


@pytest.mark.parametrize("scale", [1e-6, 1e6])
def test_scale_invariance_fp32(qlib, scale):
    rng = synth.config_rng(1)
    x, _ = synth.line_1d_scatterers(rng, 2 ** 13, nscat=20, snr_db=20.0)
    xs = (x * scale).astype(np.complex64)
    _, _, out = _pipeline(qlib, xs, 128.0, 0.0, 32, 1e-7, 1e-7)
    ref = P.conv_sinc_qtt(xs.astype(np.complex128), 128.0, 0.0, 32, eps_op=1e-7, eps_round=1e-7)
    assert C.rel_l2(out.astype(np.complex128), ref) <= 1e-5


# ------------------------------------------------------------- argument errors
def test_argument_errors_are_status_codes(qlib):
    import torch
    q = qlib
    L = q.lib()
    x = torch.zeros(2 ** 8, dtype=torch.complex64, device="cuda")
    with pytest.raises(ValueError):
        q.qtt_decompose(torch.zeros(100, dtype=torch.complex64, device="cuda"))
    out = ctypes.c_void_p()
    tr = q._trunc(0.0, 8, True)
    bad_shape = (ctypes.c_int * 2)(0, 0)
    st = L.qtt_decompose(ctypes.c_void_p(x.data_ptr()), q.QTT_C64, 1, bad_shape, 1,
                         ctypes.byref(tr), q._stream(None), ctypes.byref(out))
    assert st == -1 and b"log2" in L.qtt_last_error()
    tr_bad = q._trunc(1.5, 8, True)
    good_shape = (ctypes.c_int * 2)(8, 0)
    st = L.qtt_decompose(ctypes.c_void_p(x.data_ptr()), q.QTT_C64, 1, good_shape, 1,
                         ctypes.byref(tr_bad), q._stream(None), ctypes.byref(out))
    assert st == -1
    f = q.qtt_decompose(x, eps=0.0, rmax=8)
    with pytest.raises(q.QTTError):
        q.qtt_conv_sinc(f, -3.0)
    with pytest.raises(q.QTTError):
        q.qtt_conv_sinc(f, 10.0, eps_op=0.0)
    with pytest.raises(q.QTTError):
        q.qtt_decompose(x, eps=0.0, rmax=8, delta=2.0)
    # the context stays usable after every rejected call
    torch.cuda.synchronize()
    assert f.ranks()[0] == 1
