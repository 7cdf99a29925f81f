"""GPU parity of every hot-path step against the FP64 CPU oracle (C ABI).

Tolerances (relative l2, Eq. err_conv): 1e-12 for the FP64 path (QTT_F64),
1e-5 for the FP32 path (QTT_C64); TT ranks decided by the GPU must equal the
oracle's (integer decisions, bit-exact).
"""
import numpy as np
import pytest

from oracle import qtt as Q, conv as C, toeplitz as T, pipeline as P
import synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


def _torch():
    import torch
    return torch


def _to_dev(x):
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _rand_cores(rng, d, r, dtype):
    ranks = [1] + [min(r, 2 ** k, 2 ** (d - k)) for k in range(1, d)] + [1]
    cores = []
    for k in range(d):
        shp = (ranks[k], 2, ranks[k + 1])
        c = rng.standard_normal(shp)
        if dtype == np.complex64:
            c = c + 1j * rng.standard_normal(shp)
        cores.append((c / np.sqrt(2 * ranks[k])).astype(dtype))
    return cores


# ------------------------------------------------------------------ a7 Full
@pytest.mark.parametrize("dtype,d", [(np.float64, 10), (np.complex64, 11), (np.complex64, 13)])
def test_full_1d(qlib, dtype, d):
    rng = np.random.default_rng(1)
    cores = _rand_cores(rng, d, 12, dtype)
    t = qlib.qtt_from_cores(cores, [d])
    out = qlib.qtt_to_full(t).cpu().numpy()
    ref = Q.full([c.astype(np.complex128 if dtype == np.complex64 else np.float64) for c in cores])
    tol = TOL64 if dtype == np.float64 else TOL32
    assert C.rel_l2(out, ref) <= tol


@pytest.mark.parametrize("interleave", [True, False])
@pytest.mark.parametrize("dy,dx", [(5, 5), (6, 6), (3, 5)])
def test_full_2d(qlib, interleave, dy, dx):
    rng = np.random.default_rng(2)
    d = dx + dy
    cores = _rand_cores(rng, d, 9, np.complex64)
    t = qlib.qtt_from_cores(cores, [dy, dx], interleave=interleave)
    out = qlib.qtt_to_full(t).cpu().numpy()
    v = Q.full([c.astype(np.complex128) for c in cores])
    ref = Q.qtt_vector_to_image(v, 2 ** dy, 2 ** dx, interleave)
    assert out.shape == ref.shape
    assert C.rel_l2(out, ref) <= TOL32


# ------------------------------------------------------------------ a2/a3 TT-SVD
def test_decompose_fp64_config1_like(qlib):
    rng = synth.config_rng(0)
    x, _ = synth.line_1d_bumps(rng, 4096)
    t = qlib.qtt_decompose(_to_dev(x), eps=1e-2, rmax=0, refine=True)
    ranks = t.ranks()
    cores, oranks, _ = Q.tt_svd(x, 12, 1e-2)
    assert ranks == oranks
    out = qlib.qtt_to_full(t).cpu().numpy()
    assert C.rel_l2(out, Q.full(cores)) <= TOL64


@pytest.mark.parametrize("refine", [False, True])
def test_decompose_c64_capped(qlib, refine):
    rng = synth.config_rng(1)
    x, _ = synth.line_1d_scatterers(rng, 2 ** 14, nscat=30, snr_db=20.0)
    x = x.astype(np.complex64)
    t = qlib.qtt_decompose(_to_dev(x), eps=0.0, rmax=32, refine=refine)
    cores, oranks, _ = Q.tt_svd(x.astype(np.complex128), 14, 0.0, 32)
    assert t.ranks() == oranks
    out = qlib.qtt_to_full(t).cpu().numpy().astype(np.complex128)
    # one FP32 Gram pass squares the condition of the cut inside the noise
    # cluster (eigenvector error ~ u lambda_1 / gap); the refined path is the
    # one held to the FP32 tolerance
    assert C.rel_l2(out, Q.full(cores)) <= (TOL32 if refine else 1e-4)


def test_decompose_2d_interleaved(qlib):
    rng = synth.config_rng(2)
    x, _ = synth.image_2d_scene(rng, 64, 64, nscat=10, nrect=2, rect_min=4, rect_max=16)
    x = x.astype(np.complex64)
    t = qlib.qtt_decompose(_to_dev(x), eps=3e-2, rmax=16, refine=True, interleave=True)
    cores, oranks, _ = P.decompose(x.astype(np.complex128), 3e-2, 16, interleave=True)
    assert t.ranks() == oranks
    out = qlib.qtt_to_full(t).cpu().numpy().astype(np.complex128)
    ref = Q.qtt_vector_to_image(Q.full(cores), 64, 64, True)
    assert C.rel_l2(out, ref) <= TOL32


def test_decompose_exact_lowrank(qlib):
    # exponential: QTT rank 1 exactly; untruncated reconstruction is exact
    d = 12
    x = np.exp(0.37 * np.arange(2 ** d) / 2 ** d)
    t = qlib.qtt_decompose(_to_dev(x), eps=1e-10, rmax=0, refine=True)
    assert max(t.ranks()) == 1
    out = qlib.qtt_to_full(t).cpu().numpy()
    assert C.rel_l2(out, x) <= TOL64


# ------------------------------------------------------------------ a4 operator
@pytest.mark.parametrize("d,B", [(8, 16.0), (9, 40.0)])
def test_operator_dense_fp64(qlib, d, B):
    op = qlib.qtt_op_create(d, B, True, 1e-13, qlib.QTT_F64)
    Tq = T.operator_dense(op.cores())
    Tref = C.toeplitz_dense(C.sinc_taps(2 ** d, B, True))
    assert np.abs(Tq - Tref).max() <= 1e-12 * np.abs(Tref).max() * 2 ** (d / 2)
    ops_o = T.toeplitz_qtt(C.sinc_taps(2 ** d, B, True), 1e-13)
    assert op.ranks() == [1] + [o.shape[3] for o in ops_o]


# ------------------------------------------------------------------ a5 matvec
def test_matvec_fp64(qlib):
    d, B = 9, 24.0
    rng = np.random.default_rng(3)
    cores = _rand_cores(rng, d, 6, np.float64)
    t = qlib.qtt_from_cores(cores, [d])
    op = qlib.qtt_op_create(d, B, True, 1e-13, qlib.QTT_F64)
    y = qlib.qtt_matvec(op, t)
    out = qlib.qtt_to_full(y).cpu().numpy()
    ref = C.conv_direct(Q.full(cores), C.sinc_taps(2 ** d, B, True))
    assert C.rel_l2(out, ref) <= 1e-11


# ------------------------------------------------------------------ a6 rounding
def test_round_fp64(qlib):
    d, B = 10, 32.0
    rng = np.random.default_rng(4)
    cores = _rand_cores(rng, d, 5, np.float64)
    t = qlib.qtt_from_cores(cores, [d])
    op = qlib.qtt_op_create(d, B, True, 1e-13, qlib.QTT_F64)
    y = qlib.qtt_matvec(op, t)
    qlib.qtt_round(y, 1e-10, sketch=64)
    out = qlib.qtt_to_full(y).cpu().numpy()
    ops_o = T.toeplitz_qtt(C.sinc_taps(2 ** d, B, True), 1e-13)
    Yo = Q.tt_round(T.matvec(ops_o, cores), 1e-10)
    assert C.rel_l2(out, Q.full(Yo)) <= 1e-9


# ------------------------------------------------------------------ pipeline
def test_pipeline_config1_fp64(qlib):
    rng = synth.config_rng(0)
    x, _ = synth.line_1d_bumps(rng, 4096)
    f = qlib.qtt_decompose(_to_dev(x), eps=1e-2, rmax=0, refine=True)
    y = qlib.qtt_conv_sinc(f, 64.0, eps_op=1e-12, eps_round=1e-12, sketch=64)
    out = qlib.qtt_to_full(y).cpu().numpy()
    ref = P.conv_sinc_qtt(x, 64.0, 1e-2, None, eps_op=1e-12, eps_round=1e-12)
    assert C.rel_l2(out, ref) <= TOL64


def test_pipeline_c64_1d(qlib):
    rng = synth.config_rng(1)
    d = 14
    x, _ = synth.line_1d_scatterers(rng, 2 ** d, nscat=30, snr_db=20.0)
    x = x.astype(np.complex64)
    B = 1024.0 * 2 ** d / 2 ** 20
    f = qlib.qtt_decompose(_to_dev(x), eps=0.0, rmax=64, refine=True)
    y = qlib.qtt_conv_sinc(f, B, eps_op=1e-7, eps_round=1e-7)
    out = qlib.qtt_to_full(y).cpu().numpy().astype(np.complex128)
    ref = P.conv_sinc_qtt(x.astype(np.complex128), B, 0.0, 64, eps_op=1e-7, eps_round=1e-7)
    assert C.rel_l2(out, ref) <= TOL32


@pytest.mark.parametrize("n", [16, 32])
def test_pipeline_c64_2d(qlib, n):
    # sizes whose rounding ranks stay below the sketch capacity
    rng = synth.config_rng(2)
    x, _ = synth.image_2d_scene(rng, n, n, nscat=10, nrect=2, rect_min=4, rect_max=16)
    x = x.astype(np.complex64)
    B = 256.0 * n / 4096
    f = qlib.qtt_decompose(_to_dev(x), eps=3e-2, rmax=64, refine=True)
    y = qlib.qtt_conv_sinc(f, [B, B], eps_op=1e-7, eps_round=1e-7)
    out = qlib.qtt_to_full(y).cpu().numpy().astype(np.complex128)
    ref = P.conv_sinc_qtt(x.astype(np.complex128), B, 3e-2, 64, eps_op=1e-7, eps_round=1e-7)
    assert C.rel_l2(out, ref) <= TOL32


@pytest.mark.parametrize("dtype,noise,delta,tol", [(np.float64, 1e-9, 1e-3, 1e-12),
                                                    (np.complex64, 1e-4, 1e-2, 1e-5)])
def test_decompose_sv_dropoff(qlib, dtype, noise, delta, tol):
    """Sec. 5 modification (3): ranks and reconstruction equal the oracle's."""
    import torch
    q = qlib
    rng = np.random.default_rng(17)
    d = 12
    i = np.arange(2 ** d)
    v = np.exp(-i / 700.0) + 0.5 * np.exp(-i / 90.0) + 0.25 * np.cos(i / 33.0)
    if dtype == np.complex64:
        v = v * np.exp(1j * i / 50.0)
    v = v + noise * np.linalg.norm(v) / np.sqrt(v.size) * rng.standard_normal(v.size)
    x = v.astype(dtype)
    cores, ranks, _ = P.decompose(x.astype(np.complex128 if dtype == np.complex64 else np.float64),
                                  0.0, None, delta=delta)
    t = q.qtt_decompose(torch.from_numpy(x).cuda(), eps=0.0, rmax=0, refine=True, delta=delta)
    assert t.ranks() == ranks
    got = q.qtt_to_full(t).cpu().numpy()
    assert C.rel_l2(got, Q.full(cores)) <= tol
