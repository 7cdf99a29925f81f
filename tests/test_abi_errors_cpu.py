"""Argument errors of the C ABI, without a GPU: every call below is rejected
by the entry point's own checks before any CUDA call, returns QTT_EINVAL
(-1) and leaves a message for qtt_last_error.  The buffers passed are host
memory that the rejected calls never touch."""
import ctypes

import pytest

QTT_EINVAL = -1
QTT_EUNSUPPORTED = -6
QTT_F64, QTT_F32, QTT_C64, QTT_C128 = 0, 1, 2, 3


class Trunc(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("rmax", ctypes.c_int), ("refine", ctypes.c_int),
                ("delta", ctypes.c_double), ("prec", ctypes.c_int),
                ("fixed_ranks", ctypes.POINTER(ctypes.c_int))]


@pytest.fixture(scope="module")
def lib():
    from paper_2301_13339_gb300 import _build
    L = ctypes.CDLL(_build.build())
    L.qtt_last_error.restype = ctypes.c_char_p
    return L


@pytest.fixture
def buf():
    return ctypes.create_string_buffer(4096)


def _expect(lib, status, words, code=QTT_EINVAL):
    assert status == code
    msg = lib.qtt_last_error().decode()
    for w in words:
        assert w in msg, msg


def test_decompose_arguments(lib, buf):
    out = ctypes.c_void_p()
    ok = Trunc(0.0, 64, 1, 0.0)
    sh = (ctypes.c_int * 2)(10, 0)
    p = ctypes.cast(buf, ctypes.c_void_p)
    f = lib.qtt_decompose
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                  ctypes.c_int, ctypes.POINTER(Trunc), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    _expect(lib, f(None, QTT_C64, 1, sh, 1, ctypes.byref(ok), None, ctypes.byref(out)), ["NULL"])
    _expect(lib, f(p, 7, 1, sh, 1, ctypes.byref(ok), None, ctypes.byref(out)), ["dtype"])
    for dt in (QTT_F32, QTT_C128):   # named by the ABI, not built
        _expect(lib, f(p, dt, 1, sh, 1, ctypes.byref(ok), None, ctypes.byref(out)),
                ["not built"], QTT_EUNSUPPORTED)
    # precision selector: the BF16-refined mode is not built, the TF32-refined
    # one only for complex64; FP64 with complex64 data
    _expect(lib, f(p, QTT_C64, 1, sh, 1, ctypes.byref(Trunc(0.0, 64, 1, 0.0, 3, None)), None,
                   ctypes.byref(out)), ["not built"], QTT_EUNSUPPORTED)
    _expect(lib, f(p, QTT_F64, 1, sh, 1, ctypes.byref(Trunc(0.0, 64, 1, 0.0, 4, None)), None,
                   ctypes.byref(out)), ["complex64"], QTT_EUNSUPPORTED)
    _expect(lib, f(p, QTT_C64, 1, sh, 1, ctypes.byref(Trunc(0.0, 64, 1, 0.0, 1, None)), None,
                   ctypes.byref(out)), ["does not match"])
    _expect(lib, f(p, QTT_F64, 1, sh, 1, ctypes.byref(Trunc(0.0, 64, 1, 0.0, 2, None)), None,
                   ctypes.byref(out)), ["does not match"])
    _expect(lib, f(p, QTT_C64, 1, sh, 1, ctypes.byref(Trunc(0.0, 64, 1, 0.0, 9, None)), None,
                   ctypes.byref(out)), ["qtt_prec"])
    # forced ranks: ends not 1, a rank above min(2^k, 2^(d-k), 64)
    bad_ends = (ctypes.c_int * 11)(*([2] + [1] * 9 + [1]))
    too_big = (ctypes.c_int * 11)(1, 2, 4, 9, 16, 32, 16, 8, 4, 2, 1)
    for fr, w in ((bad_ends, "r_0"), (too_big, "r_3")):
        tr = Trunc(0.0, 0, 1, 0.0, 0, ctypes.cast(fr, ctypes.POINTER(ctypes.c_int)))
        _expect(lib, f(p, QTT_C64, 1, sh, 1, ctypes.byref(tr), None, ctypes.byref(out)), [w])
    _expect(lib, f(p, QTT_C64, 3, sh, 1, ctypes.byref(ok), None, ctypes.byref(out)), ["ndim"])
    _expect(lib, f(p, QTT_C64, 1, sh, 1, None, None, ctypes.byref(out)), ["NULL"])
    _expect(lib, f(p, QTT_C64, 1, sh, 1, ctypes.byref(Trunc(1.5, 0, 1, 0.0)), None,
                   ctypes.byref(out)), ["eps"])
    _expect(lib, f(p, QTT_C64, 1, sh, 1, ctypes.byref(Trunc(0.0, 0, 1, 1.0)), None,
                   ctypes.byref(out)), ["delta"])
    _expect(lib, f(p, QTT_C64, 1, (ctypes.c_int * 2)(31, 0), 1, ctypes.byref(ok), None,
                   ctypes.byref(out)), ["out of range"])
    _expect(lib, f(p, QTT_C64, 1, (ctypes.c_int * 2)(1, 0), 1, ctypes.byref(ok), None,
                   ctypes.byref(out)), ["d=1"])
    assert not out.value


def test_rsvd_arguments(lib, buf):
    out = ctypes.c_void_p()
    p = ctypes.cast(buf, ctypes.c_void_p)
    f = lib.qtt_decompose_rsvd
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_ulonglong, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    _expect(lib, f(p, QTT_C64, 10, 0, 4, None, 1, None, ctypes.byref(out)), ["rmax"])
    _expect(lib, f(p, QTT_C64, 10, 64, 40, None, 1, None, ctypes.byref(out)), ["rmax + p"])
    _expect(lib, f(p, QTT_C64, 10, 8, 0, None, 1, None, ctypes.byref(out)), ["p >= 1"])
    _expect(lib, f(p, QTT_C64, 1, 8, 4, None, 1, None, ctypes.byref(out)), ["log2 length"])
    assert not out.value


def test_sinc_padded_arguments(lib, buf):
    p = ctypes.cast(buf, ctypes.c_void_p)
    f = lib.qtt_sinc_padded
    f.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_void_p]
    _expect(lib, f(10, 511, 64.0, 1, QTT_C64, None, None), ["NULL"])
    _expect(lib, f(10, 510, 64.0, 1, QTT_C64, p, None), ["N odd"])      # even N
    _expect(lib, f(10, 513, 64.0, 1, QTT_C64, p, None), ["N odd"])      # 2N - 1 > n
    _expect(lib, f(10, 0, 64.0, 1, QTT_C64, p, None), ["N odd"])
    _expect(lib, f(31, 511, 64.0, 1, QTT_C64, p, None), ["log2_n"])
    _expect(lib, f(10, 511, 64.0, 1, 7, p, None), ["dtype"])
    _expect(lib, f(10, 511, 64.0, 1, QTT_C128, p, None), ["not built"], QTT_EUNSUPPORTED)


def test_handle_entries_reject_null(lib, buf):
    out = ctypes.c_void_p()
    p = ctypes.cast(buf, ctypes.c_void_p)
    lib.qtt_fft.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(Trunc), ctypes.c_int,
                            ctypes.c_ulonglong, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    _expect(lib, lib.qtt_fft(None, 0, None, 0, 1, None, ctypes.byref(out)), ["qtt_fft", "NULL"])
    lib.qtt_hadamard.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.POINTER(ctypes.c_void_p)]
    _expect(lib, lib.qtt_hadamard(None, None, None, ctypes.byref(out)), ["qtt_hadamard", "NULL"])
    lib.qtt_to_full.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    _expect(lib, lib.qtt_to_full(None, p, None), ["qtt_to_full", "NULL"])
    lib.qtt_conv_sinc.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                  ctypes.c_double, ctypes.POINTER(Trunc), ctypes.c_int,
                                  ctypes.c_ulonglong, ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_void_p)]
    _expect(lib, lib.qtt_conv_sinc(None, None, 1, 1e-7, None, 0, 1, None, ctypes.byref(out)),
            ["qtt_conv_sinc", "NULL"])
    assert not out.value


def test_from_cores_and_operator_arguments(lib, buf):
    out = ctypes.c_void_p()
    p = ctypes.cast(buf, ctypes.c_void_p)
    f = lib.qtt_from_cores
    f.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                  ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_void_p,
                  ctypes.POINTER(ctypes.c_void_p)]
    sh = (ctypes.c_int * 2)(4, 0)
    _expect(lib, f(p, (ctypes.c_int * 5)(2, 2, 2, 2, 1), 4, QTT_C64, 1, sh, 1, None,
                   ctypes.byref(out)), ["boundary ranks"])
    _expect(lib, f(p, (ctypes.c_int * 5)(1, 2, 2, 2, 1), 4, QTT_C64, 1, (ctypes.c_int * 2)(5, 0), 1,
                   None, ctypes.byref(out)), ["log2 shape"])
    _expect(lib, f(p, (ctypes.c_int * 5)(1, 0, 2, 2, 1), 4, QTT_C64, 1, sh, 1, None,
                   ctypes.byref(out)), ["rank"])
    g = lib.qtt_op_create
    g.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                  ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    _expect(lib, g(10, 0.0, 1, 1e-7, QTT_C64, None, ctypes.byref(out)), ["B > 0"])
    _expect(lib, g(10, 64.0, 1, 0.0, QTT_C64, None, ctypes.byref(out)), ["eps_op"])
    assert not out.value


def test_big_qr_arguments(lib, buf):
    """qtt_debug_big_qr checks its shape, its dtype and its arrays before
    touching the device."""
    f = lib.qtt_debug_big_qr
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_void_p]
    p = ctypes.cast(buf, ctypes.c_void_p)
    _expect(lib, f(None, 8, 4, 4, QTT_C64, p, None), ["qtt_debug_big_qr"])        # NULL A
    _expect(lib, f(p, 8, 4, 4, QTT_C64, None, None), ["qtt_debug_big_qr"])        # NULL Q
    _expect(lib, f(p, 1025, 4, 4, QTT_C64, p, None), ["1025"])                    # above 1024 rows
    _expect(lib, f(p, 8, 4, 9, QTT_C64, p, None), ["nq 9"])                       # nq > m
    _expect(lib, f(p, 8, 0, 4, QTT_C64, p, None), ["qtt_debug_big_qr"])           # no columns
    _expect(lib, f(p, 8, 4, 4, QTT_F32, p, None), ["dtype 1"])                    # not built
