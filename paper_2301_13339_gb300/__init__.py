"""GB300 QTT denoising convolution (arXiv 2301.13339) -- Python binding.

Thin ctypes marshalling over ``libqtt.so`` (the C ABI in ``include/qtt.h``):
every step of the computation runs in the library's CUDA kernels.  PyTorch
provides device memory and streams only.  If the compiled library is missing
the import fails; there is no CPU fallback.

The functions carry the names of the C entry points:
``qtt_decompose``, ``qtt_conv_sinc``, ``qtt_round``, ``qtt_to_full``,
``qtt_conv_adjoint``, ``qtt_matvec``, ``qtt_op_create`` ...
"""
import ctypes
import os

import numpy as np

from . import _build

__all__ = [
    "QTTError", "QTTTensor", "QTTOperator", "lib", "load", "qtt_decompose", "qtt_conv_sinc",
    "qtt_round", "qtt_to_full", "qtt_to_full_noalloc", "qtt_conv_adjoint", "qtt_matvec",
    "qtt_op_create",
    "qtt_from_cores", "big_qr", "QTT_F64", "QTT_C64", "QTT_RANK_CAP", "QTT_SKETCH_CAP_BIG", "EXPORTED_SYMBOLS",
    "QTTBatch", "qtt_batch_conv_sinc", "autotune_batch", "qtt_dot", "qtt_add", "qtt_core_grads",
    "qtt_from_device_cores", "empty_cores", "core_tensors", "qtt_decompose_rsvd", "qtt_fft",
    "qtt_hadamard", "qtt_conv_fft", "qtt_sinc_padded", "QTT_PREC_AUTO", "QTT_PREC_FP64",
    "QTT_PREC_FP32", "QTT_PREC_BF16_REFINED", "QTT_PREC_TF32_REFINED",
]

QTT_F64 = 0
QTT_C64 = 2
QTT_RANK_CAP = 64
QTT_SKETCH_CAP_BIG = 512

_STATUS = {0: "QTT_OK", -1: "QTT_EINVAL", -2: "QTT_ENOMEM", -3: "QTT_ECUDA",
           -4: "QTT_ETIMEOUT", -5: "QTT_ERANK", -6: "QTT_EUNSUPPORTED", -7: "QTT_ENUMERIC"}

EXPORTED_SYMBOLS = [
    "qtt_decompose", "qtt_conv_sinc", "qtt_round", "qtt_to_full", "qtt_to_full_noalloc",
    "qtt_conv_adjoint", "qtt_get_ranks", "qtt_get_info", "qtt_get_cores", "qtt_from_cores", "qtt_free",
    "qtt_free_async", "qtt_op_create", "qtt_op_get_ranks", "qtt_op_get_cores", "qtt_op_free",
    "qtt_matvec", "qtt_release_workspace", "qtt_last_error", "qtt_version", "qtt_small_eigh",
    "qtt_debug_set_eig_solver", "qtt_profile_enable", "qtt_profile_read", "qtt_profile_reset",
    "qtt_profile_work", "qtt_get_margins", "qtt_debug_tc_selftest", "qtt_debug_tc_cgemm",
    "qtt_debug_set_tc_gemm", "qtt_debug_tc_gram", "qtt_debug_set_orth_fix", "qtt_debug_set_tc_gram",
    "qtt_debug_set_proj_acc", "qtt_debug_fill_pool", "qtt_debug_set_heev_repair",
    "qtt_debug_set_env_big", "qtt_debug_big_qr",
    "qtt_core_grads", "qtt_dot", "qtt_add", "qtt_from_device_cores",
    "qtt_batch_create", "qtt_batch_run", "qtt_batch_capture", "qtt_batch_launch", "qtt_batch_info",
    "qtt_batch_free", "qtt_batch_conv_sinc", "qtt_decompose_rsvd", "qtt_fft", "qtt_hadamard",
    "qtt_sinc_padded", "qtt_batch_set_tiles",
]


class QTTError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Trunc(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("rmax", ctypes.c_int), ("refine", ctypes.c_int),
                ("delta", ctypes.c_double), ("prec", ctypes.c_int),
                ("fixed_ranks", ctypes.POINTER(ctypes.c_int))]


_lib = None


def load(path=None):
    """Load libqtt.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libqtt.so not found at {path}: run "
                          "`python -c 'import __graft_entry__ as g; g.build()'` first")
    L = ctypes.CDLL(path)
    vp, i, d, ull = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_ulonglong
    ip = ctypes.POINTER(ctypes.c_int)
    dp = ctypes.POINTER(ctypes.c_double)
    pp = ctypes.POINTER(ctypes.c_void_p)
    tp = ctypes.POINTER(_Trunc)
    sig = {
        "qtt_decompose": (i, [vp, i, i, ip, i, tp, vp, pp]),
        "qtt_conv_sinc": (i, [vp, dp, i, d, tp, i, ull, vp, pp]),
        "qtt_round": (i, [vp, tp, i, ull, vp]),
        "qtt_to_full": (i, [vp, vp, vp]),
        "qtt_to_full_noalloc": (i, [vp, vp, vp]),
        "qtt_conv_adjoint": (i, [vp, vp, dp, i, d, tp, i, ull, pp, pp, vp]),
        "qtt_core_grads": (i, [vp, vp, d, d, pp, vp]),
        "qtt_dot": (i, [vp, vp, vp, vp]),
        "qtt_add": (i, [d, vp, d, vp, vp, pp]),
        "qtt_from_device_cores": (i, [pp, ip, i, i, i, ip, i, vp, pp]),
        "qtt_batch_create": (i, [i, ip, dp, ip, d, i, i, d, tp, i, i, vp, pp]),
        "qtt_batch_run": (i, [vp, pp, pp, vp]),
        "qtt_batch_capture": (i, [vp, pp, pp, vp]),
        "qtt_batch_launch": (i, [vp, vp]),
        "qtt_batch_info": (i, [vp, ip, ip]),
        "qtt_batch_free": (None, [vp]),
        "qtt_batch_conv_sinc": (i, [i, pp, ip, dp, ip, d, i, i, d, tp, pp, i, vp]),
        "qtt_get_ranks": (i, [vp, ip, vp]),
        "qtt_get_margins": (i, [vp, dp, vp]),
        "qtt_get_info": (i, [vp, ip, ip, ip, ip, ip]),
        "qtt_get_cores": (i, [vp, vp, vp]),
        "qtt_from_cores": (i, [vp, ip, i, i, i, ip, i, vp, pp]),
        "qtt_free": (None, [vp]),
        "qtt_free_async": (None, [vp, vp]),
        "qtt_op_create": (i, [i, d, i, d, i, vp, pp]),
        "qtt_op_get_ranks": (i, [vp, ip]),
        "qtt_op_get_cores": (i, [vp, vp]),
        "qtt_op_free": (None, [vp]),
        "qtt_matvec": (i, [vp, vp, vp, pp]),
        "qtt_fft": (i, [vp, i, tp, i, ull, vp, pp]),
        "qtt_hadamard": (i, [vp, vp, vp, pp]),
        "qtt_sinc_padded": (i, [i, ctypes.c_longlong, d, i, i, vp, vp]),
        "qtt_release_workspace": (None, []),
        "qtt_small_eigh": (i, [vp, i, i, vp, vp, vp]),
        "qtt_debug_set_eig_solver": (None, [i]),
        "qtt_debug_set_heev_cluster": (None, [d, i]),
        "qtt_decompose_rsvd": (i, [vp, i, i, i, i, vp, ctypes.c_ulonglong, vp, pp]),
        "qtt_debug_set_refine_sweeps": (None, [i]),
        "qtt_debug_big_qr": (i, [vp, i, i, i, i, vp, vp]),
        "qtt_last_error": (ctypes.c_char_p, []),
        "qtt_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def lib():
    return load()


def _check(st):
    if st != 0:
        raise QTTError(st, _lib.qtt_last_error().decode())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_code(t):
    import torch
    if t.dtype == torch.float64:
        return QTT_F64
    if t.dtype == torch.complex64:
        return QTT_C64
    raise TypeError(f"unsupported dtype {t.dtype}: use torch.float64 or torch.complex64")


def _np_dtype(code):
    return np.float64 if code == QTT_F64 else np.complex64


class QTTTensor:
    """Library-owned QTT tensor (device cores, device ranks)."""

    def __init__(self, handle):
        self._h = ctypes.c_void_p(handle) if not isinstance(handle, ctypes.c_void_p) else handle
        d = ctypes.c_int()
        dt = ctypes.c_int()
        nd = ctypes.c_int()
        sh = (ctypes.c_int * 2)()
        il = ctypes.c_int()
        _check(_lib.qtt_get_info(self._h, ctypes.byref(d), ctypes.byref(dt), ctypes.byref(nd), sh,
                                 ctypes.byref(il)))
        self.d = d.value
        self.dtype_code = dt.value
        self.ndim = nd.value
        self.log2_shape = tuple(sh[k] for k in range(self.ndim))
        self.interleave = il.value

    @property
    def handle(self):
        return self._h

    @property
    def shape(self):
        return tuple(1 << s for s in self.log2_shape)

    def ranks(self, stream=None):
        r = (ctypes.c_int * (self.d + 1))()
        _check(_lib.qtt_get_ranks(self._h, r, _stream(stream)))
        return [r[k] for k in range(self.d + 1)]

    def margins(self, stream=None):
        """Per-cut margin of the eps-rank decisions (qtt_get_margins; NaN
        where no eps rule decided)."""
        m = (ctypes.c_double * (self.d + 1))()
        _check(_lib.qtt_get_margins(self._h, m, _stream(stream)))
        return [m[k] for k in range(self.d + 1)]

    def cores(self, stream=None):
        """Cores as numpy arrays of shape (r_{k-1}, 2, r_k) (host copies)."""
        r = self.ranks(stream)
        n = sum(r[k] * 2 * r[k + 1] for k in range(self.d))
        buf = np.empty(n, dtype=_np_dtype(self.dtype_code))
        _check(_lib.qtt_get_cores(self._h, buf.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
        out, o = [], 0
        for k in range(self.d):
            c = r[k] * 2 * r[k + 1]
            out.append(buf[o:o + c].reshape((r[k], 2, r[k + 1]), order="F").copy())
            o += c
        return out

    def free(self, stream=None):
        if self._h is not None and self._h.value:
            if stream is None:
                _lib.qtt_free(self._h)
            else:
                _lib.qtt_free_async(self._h, _stream(stream))
        self._h = None

    def __del__(self):
        try:
            if _lib is not None and self._h is not None and self._h.value:
                _lib.qtt_free(self._h)
        except Exception:
            pass


class QTTOperator:
    def __init__(self, handle, d, dtype_code):
        self._h = handle
        self.d = d
        self.dtype_code = dtype_code

    def ranks(self):
        r = (ctypes.c_int * (self.d + 1))()
        _check(_lib.qtt_op_get_ranks(self._h, r))
        return [r[k] for k in range(self.d + 1)]

    def cores(self):
        """Cores as numpy arrays O[p, j, i, q] of shape (P_{k-1}, 2, 2, P_k)."""
        P = self.ranks()
        n = sum(P[k] * 4 * P[k + 1] for k in range(self.d))
        buf = np.empty(n, dtype=np.float64 if self.dtype_code == QTT_F64 else np.float32)
        _check(_lib.qtt_op_get_cores(self._h, buf.ctypes.data_as(ctypes.c_void_p)))
        out, o = [], 0
        for k in range(self.d):
            c = P[k] * 4 * P[k + 1]
            out.append(buf[o:o + c].reshape((P[k], 2, 2, P[k + 1]), order="F").copy())
            o += c
        return out

    def __del__(self):
        try:
            if _lib is not None and self._h is not None and self._h.value:
                _lib.qtt_op_free(self._h)
        except Exception:
            pass


QTT_PREC_AUTO, QTT_PREC_FP64, QTT_PREC_FP32, QTT_PREC_BF16_REFINED, QTT_PREC_TF32_REFINED = range(5)


def _trunc(eps, rmax, refine, delta=0.0, prec=QTT_PREC_AUTO, fixed_ranks=None):
    """qtt_trunc.  fixed_ranks: None or the d+1 ranks r_0..r_d to force (the
    array is kept alive on the returned structure)."""
    tr = _Trunc(float(eps), int(rmax or 0), int(bool(refine)), float(delta or 0.0), int(prec), None)
    if fixed_ranks is not None:
        arr = (ctypes.c_int * len(fixed_ranks))(*[int(r) for r in fixed_ranks])
        tr.fixed_ranks = ctypes.cast(arr, ctypes.POINTER(ctypes.c_int))
        tr._keep = arr
    return tr


def qtt_decompose(x, eps=0.0, rmax=0, refine=False, interleave=True, stream=None, delta=0.0,
                  prec=QTT_PREC_AUTO, fixed_ranks=None):
    """QTT reshape + TT-SVD (Alg. 1 with the max-rank cap of Sec. 5) of a
    contiguous CUDA tensor (1D length 2^d, or 2D 2^dy x 2^dx row-major).
    delta > 0: the SV drop-off rule (Sec. 5 (3)) instead of eps.
    fixed_ranks: the d+1 ranks to keep (parity mode; eps/rmax/delta unused)."""
    load()
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError("x must be a contiguous CUDA tensor")
    code = _dtype_code(x)
    shape = []
    for n in x.shape:
        ln = int(n).bit_length() - 1
        if n < 2 or (1 << ln) != n:
            raise ValueError(f"sizes must be powers of two >= 2, got {tuple(x.shape)}")
        shape.append(ln)
    sh = (ctypes.c_int * 2)(*(shape + [0] * (2 - len(shape))))
    tr = _trunc(eps, rmax, refine, delta, prec, fixed_ranks)
    out = ctypes.c_void_p()
    _check(_lib.qtt_decompose(ctypes.c_void_p(x.data_ptr()), code, x.dim(), sh, int(interleave),
                              ctypes.byref(tr), _stream(stream), ctypes.byref(out)))
    return QTTTensor(out)


def qtt_decompose_rsvd(x, rmax, p, omega=None, seed=20230131, stream=None):
    """Max rank TT-RSVD (Sec. 5 modification (2), App. A Algs. 4-5) of a
    contiguous 1D CUDA tensor of length 2^d.  omega: None (Gaussian test
    matrices drawn on the device from seed) or a contiguous CUDA tensor of
    the real dtype (float32 for complex64 x, float64 for float64 x) holding
    the n_k x (rmax + p) block of every level k = 1..d-1 column-major, one
    after the other (n_k = 2^(d-k))."""
    load()
    if not x.is_cuda or not x.is_contiguous() or x.dim() != 1:
        raise ValueError("x must be a contiguous 1D CUDA tensor")
    code = _dtype_code(x)
    n = x.shape[0]
    d = int(n).bit_length() - 1
    if n < 4 or (1 << d) != n:
        raise ValueError(f"length must be a power of two >= 4, got {n}")
    optr = None
    if omega is not None:
        import torch
        want = torch.float64 if code == QTT_F64 else torch.float32
        need = sum((1 << (d - k)) * (rmax + p) for k in range(1, d))
        if (not omega.is_cuda or not omega.is_contiguous() or omega.dtype != want
                or omega.numel() < need):
            raise ValueError(f"omega must be a contiguous CUDA {want} tensor of >= {need} elements")
        optr = ctypes.c_void_p(omega.data_ptr())
    out = ctypes.c_void_p()
    _check(_lib.qtt_decompose_rsvd(ctypes.c_void_p(x.data_ptr()), code, d, int(rmax), int(p), optr,
                                   ctypes.c_ulonglong(int(seed)), _stream(stream),
                                   ctypes.byref(out)))
    return QTTTensor(out)


def qtt_conv_sinc(f, B, normalize=True, eps_op=1e-7, eps_round=1e-7, rround=0, refine=True,
                  sketch=0, seed=20230131, stream=None, prec=QTT_PREC_AUTO, fixed_ranks=None):
    """QTT Toeplitz convolution with the sinc kernel + TT-rounding (sketch >
    QTT_RANK_CAP: the large-rank mode, see include/qtt.h)."""
    load()
    Bs = [float(B)] * f.ndim if np.isscalar(B) else [float(b) for b in B]
    Barr = (ctypes.c_double * 2)(*(Bs + [0.0] * (2 - len(Bs))))
    tr = _trunc(eps_round, rround, refine, 0.0, prec, fixed_ranks)
    out = ctypes.c_void_p()
    _check(_lib.qtt_conv_sinc(f.handle, Barr, int(bool(normalize)), float(eps_op),
                              ctypes.byref(tr), int(sketch), int(seed), _stream(stream),
                              ctypes.byref(out)))
    return QTTTensor(out)


def qtt_round(t, eps, rmax=0, refine=True, sketch=0, seed=20230131, stream=None,
              prec=QTT_PREC_AUTO, fixed_ranks=None):
    load()
    tr = _trunc(eps, rmax, refine, 0.0, prec, fixed_ranks)
    _check(_lib.qtt_round(t.handle, ctypes.byref(tr), int(sketch), int(seed), _stream(stream)))
    return t


def qtt_to_full(t, out=None, stream=None):
    """Full (Alg. 3) into a new (or the given) CUDA tensor of the input's shape."""
    import torch
    load()
    dt = torch.float64 if t.dtype_code == QTT_F64 else torch.complex64
    if out is None:
        out = torch.empty(t.shape, dtype=dt, device="cuda")
    if out.dtype != dt or tuple(out.shape) != t.shape or not out.is_contiguous():
        raise ValueError("out has the wrong dtype/shape or is not contiguous")
    _check(_lib.qtt_to_full(t.handle, ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def qtt_to_full_noalloc(t, out, stream=None):
    """Full into the caller's CUDA tensor ``out`` without any device
    allocation by the library (scratch is a static device array; calls that
    overlap on the GPU must be serialised by the caller)."""
    import torch
    load()
    dt = torch.float64 if t.dtype_code == QTT_F64 else torch.complex64
    if out.dtype != dt or tuple(out.shape) != t.shape or not out.is_contiguous():
        raise ValueError("out has the wrong dtype/shape or is not contiguous")
    _check(_lib.qtt_to_full_noalloc(t.handle, ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def _grad_ptrs(grad_cores, d):
    if grad_cores is None:
        return None
    if len(grad_cores) != d:
        raise ValueError(f"need {d} gradient buffers, got {len(grad_cores)}")
    for g in grad_cores:
        if not g.is_cuda or not _colmajor(g):
            raise ValueError("gradient buffers must be CUDA tensors (r0, 2, r1) in column-major storage")
    return (ctypes.c_void_p * d)(*[g.data_ptr() for g in grad_cores])


def _colmajor(c):
    """True when the (r0, 2, r1) tensor c is stored column-major (r0 fastest)."""
    return c.dim() == 3 and c.permute(2, 1, 0).is_contiguous()


def qtt_conv_adjoint(f, r, B, normalize=True, eps_op=1e-7, eps_round=1e-7, rround=0,
                     refine=True, sketch=0, seed=20230131, grad_cores=None, want_adj=True,
                     stream=None):
    """round(T^H r) and, if ``grad_cores`` (d CUDA tensors in f's core shapes,
    column-major) is given, the core gradients 2 dL/dconj(F_k) of
    L = ||T full(f) - g||^2 for the residual r = T f - g in QTT."""
    load()
    Bs = [float(B)] * r.ndim if np.isscalar(B) else [float(b) for b in B]
    Barr = (ctypes.c_double * 2)(*(Bs + [0.0] * (2 - len(Bs))))
    tr = _trunc(eps_round, rround, refine)
    adj = ctypes.c_void_p()
    gp = _grad_ptrs(grad_cores, r.d)
    _check(_lib.qtt_conv_adjoint(f.handle if f is not None else None, r.handle, Barr,
                                 int(bool(normalize)), float(eps_op), ctypes.byref(tr), int(sketch),
                                 int(seed), gp, ctypes.byref(adj) if want_adj else None,
                                 _stream(stream)))
    return QTTTensor(adj) if (want_adj and adj.value) else None


def qtt_core_grads(f, w, grad_cores, alpha=1.0, beta=0.0, stream=None):
    """grad_k = alpha * C_k(f, w) + beta * grad_k (chain rule through Full)."""
    load()
    gp = _grad_ptrs(grad_cores, f.d)
    _check(_lib.qtt_core_grads(f.handle, w.handle, float(alpha), float(beta), gp, _stream(stream)))
    return grad_cores


def qtt_dot(x, y, out=None, stream=None):
    """<x, y> = sum conj(x) y as a CUDA float64 tensor [re, im] (no sync)."""
    import torch
    load()
    if out is None:
        out = torch.empty(2, dtype=torch.float64, device="cuda")
    _check(_lib.qtt_dot(x.handle, y.handle, ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def qtt_add(alpha, x, beta, y, stream=None):
    """alpha x + beta y as a new handle (TT sum, ranks add; not rounded)."""
    load()
    out = ctypes.c_void_p()
    _check(_lib.qtt_add(float(alpha), x.handle, float(beta), y.handle, _stream(stream),
                        ctypes.byref(out)))
    return QTTTensor(out)


def qtt_from_device_cores(cores, shape_log2, interleave=True, stream=None):
    """Handle holding copies of CUDA core tensors (r_{k-1}, 2, r_k), each in
    column-major storage (see ``core_tensors``)."""
    import torch
    load()
    d = len(cores)
    code = _dtype_code(cores[0])
    for c in cores:
        if not c.is_cuda or not _colmajor(c) or _dtype_code(c) != code:
            raise ValueError("cores must be CUDA tensors of one dtype in column-major storage")
    ranks = [1] + [int(c.shape[2]) for c in cores]
    r = (ctypes.c_int * (d + 1))(*ranks)
    sh = (ctypes.c_int * 2)(*(list(shape_log2) + [0] * (2 - len(shape_log2))))
    ptrs = (ctypes.c_void_p * d)(*[c.data_ptr() for c in cores])
    out = ctypes.c_void_p()
    _check(_lib.qtt_from_device_cores(ptrs, r, d, code, len(shape_log2), sh, int(interleave),
                                      _stream(stream), ctypes.byref(out)))
    return QTTTensor(out)


def empty_cores(ranks, dtype, device="cuda"):
    """Uninitialised CUDA core tensors (r_{k-1}, 2, r_k) in column-major storage."""
    import torch
    return [torch.empty_strided((ranks[k], 2, ranks[k + 1]), (1, ranks[k], 2 * ranks[k]),
                                dtype=dtype, device=device) for k in range(len(ranks) - 1)]


def core_tensors(t, stream=None):
    """The cores of handle t as CUDA tensors (r_{k-1}, 2, r_k), column-major."""
    import torch
    host = t.cores(stream)
    dt = torch.float64 if t.dtype_code == QTT_F64 else torch.complex64
    out = empty_cores([1] + [c.shape[2] for c in host], dt)
    for o, c in zip(out, host):
        o.copy_(torch.from_numpy(c))
    return out


def qtt_op_create(d, B, normalize=True, eps_op=1e-7, dtype_code=QTT_C64, stream=None):
    load()
    out = ctypes.c_void_p()
    _check(_lib.qtt_op_create(int(d), float(B), int(bool(normalize)), float(eps_op),
                              int(dtype_code), _stream(stream), ctypes.byref(out)))
    return QTTOperator(out, int(d), int(dtype_code))


def qtt_matvec(op, t, stream=None):
    load()
    out = ctypes.c_void_p()
    _check(_lib.qtt_matvec(op._h, t.handle, _stream(stream), ctypes.byref(out)))
    return QTTTensor(out)


def qtt_fft(t, inverse=False, rmax=15, eps=0.0, delta=0.0, refine=True, sketch=0,
            seed=20230131, stream=None):
    """QTT-FFT (inverse=True: QTT-iFFT with its 1/N^D) of a complex64 handle
    (Sec. 4, truncated as in Sec. 5): every stage rounded to the cap rmax
    (R^_max), or with eps, or with the SV drop-off delta.  2D results are
    laid out as the transposed image (see include/qtt.h)."""
    load()
    tr = _trunc(eps, rmax, refine, delta)
    out = ctypes.c_void_p()
    _check(_lib.qtt_fft(t.handle, int(bool(inverse)), ctypes.byref(tr), int(sketch),
                        ctypes.c_ulonglong(int(seed)), _stream(stream), ctypes.byref(out)))
    return QTTTensor(out)


def qtt_sinc_padded(log2_n, N, B, normalize=True, dtype=None, out=None, stream=None):
    """The sinc kernel array g of Alg. 2, padded as in Sec. 2 (the kernel at
    the N grid points, centred, then zeros up to 2^log2_n), as a new (or the
    given) CUDA tensor of float64 or complex64."""
    import torch
    load()
    dtype = dtype or torch.complex64
    n = 1 << int(log2_n)
    if out is None:
        out = torch.empty(n, dtype=dtype, device="cuda")
    if not out.is_cuda or not out.is_contiguous() or out.numel() != n:
        raise ValueError(f"out must be a contiguous CUDA tensor of {n} elements")
    _check(_lib.qtt_sinc_padded(int(log2_n), int(N), float(B), int(bool(normalize)),
                                _dtype_code(out), ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def qtt_hadamard(x, y, stream=None):
    """Entrywise product x .* y as a new handle (ranks multiply; not rounded)."""
    load()
    out = ctypes.c_void_p()
    _check(_lib.qtt_hadamard(x.handle, y.handle, _stream(stream), ctypes.byref(out)))
    return QTTTensor(out)


def qtt_conv_fft(F, G, rhat=15, eps=0.0, delta=0.0, refine=True, stream=None):
    """Alg. 2, Step 3: QiFFT(QFFT(F) .* QFFT(G)) of two complex64 handles of
    the same layout, the transforms truncated with rhat (R^_max), eps or
    delta; the circular convolution of the two arrays, on F's layout."""
    Fh = qtt_fft(F, False, rhat, eps, delta, refine, stream=stream)
    Gh = qtt_fft(G, False, rhat, eps, delta, refine, stream=stream)
    P = qtt_hadamard(Fh, Gh, stream=stream)
    Fh.free(stream)
    Gh.free(stream)
    out = qtt_fft(P, True, rhat, eps, delta, refine, stream=stream)
    P.free(stream)
    return out


def tc_selftest(A, B, stream=None):
    """The tensor-core (tcgen05, TF32) MMA path on its own: returns
    (A @ B.T as computed on the tensor cores, wait-limit flag) for float32 CUDA
    tensors A (128 x K) and B (N x K)."""
    import torch
    load()
    N, K = int(B.shape[0]), int(B.shape[1])
    C = torch.empty((128, N), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    f = _lib.qtt_debug_tc_selftest
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    _check(f(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(C.data_ptr()),
             N, K, ctypes.c_void_p(err.data_ptr()), _stream(stream)))
    return C, int(err.item())


def tc_cgemm(A, B, conj_a=False, stream=None):
    """C = op(A) @ B (complex64 CUDA tensors, A (M x K), B (K x N)) through the
    tensor-core complex GEMM (tcgen05, 3xTF32, FP32 accumulators) of the
    large-rank rounding; returns (C, device status word)."""
    import torch
    load()
    M, K = int(A.shape[0]), int(A.shape[1])
    N = int(B.shape[1])
    if int(B.shape[0]) != K:
        raise ValueError("tc_cgemm: inner sizes differ")
    # column-major operands: the transposes of contiguous row-major copies
    Ac = A.t().contiguous()
    Bc = B.t().contiguous()
    Cc = torch.empty((N, M), dtype=torch.complex64, device=A.device)
    st = torch.zeros(1, dtype=torch.int32, device=A.device)
    f = _lib.qtt_debug_tc_cgemm
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int] * 4 + [ctypes.c_void_p, ctypes.c_void_p]
    _check(f(ctypes.c_void_p(Ac.data_ptr()), ctypes.c_void_p(Bc.data_ptr()),
             ctypes.c_void_p(Cc.data_ptr()), M, N, K, int(bool(conj_a)),
             ctypes.c_void_p(st.data_ptr()), _stream(stream)))
    return Cc.t(), int(st.item())


def tc_gram(X, split=1, max_parts=8, stream=None):
    """Per-CTA partial Grams X X^H of X (m x n complex64 CUDA tensor, m <= 128)
    on the tensor cores, as the TF32-refined TT-SVD's first pass computes
    them (split 1: TF32 operands; 3: 3xTF32).  Returns (partials as an
    (nparts, m, m) complex64 tensor, device status word)."""
    import torch
    load()
    m, n = int(X.shape[0]), int(X.shape[1])
    Xc = X.t().contiguous()                     # column-major m x n
    gp = torch.empty((max_parts, m, m), dtype=torch.complex64, device=X.device)
    st = torch.zeros(1, dtype=torch.int32, device=X.device)
    f = _lib.qtt_debug_tc_gram
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    npart = f(ctypes.c_void_p(Xc.data_ptr()), m, n, int(split), ctypes.c_void_p(gp.data_ptr()), m,
              int(max_parts), ctypes.c_void_p(st.data_ptr()), _stream(stream))
    if npart < 0:
        _check(npart)
    # element (a, b) of a partial is at a + m b: the transpose of the row-major view
    return gp[:npart].transpose(1, 2), int(st.item())


def big_qr(A, nq=None, stream=None):
    """First nq columns of Q in the blocked Householder QR A = Q R (A: m x n
    complex64 or float64 CUDA tensor, m <= 1024)."""
    import torch
    load()
    if A.dim() != 2 or A.device.type != "cuda":
        raise QTTError("big_qr: A must be a 2-D CUDA tensor")
    m, n = A.shape
    nq = m if nq is None else int(nq)
    code = {torch.complex64: QTT_C64, torch.float64: QTT_F64}.get(A.dtype)
    if code is None:
        raise QTTError("big_qr: complex64 or float64 only")
    Ac = A.t().contiguous()          # column-major
    Q = torch.empty((nq, m), dtype=A.dtype, device=A.device)
    _check(_lib.qtt_debug_big_qr(ctypes.c_void_p(Ac.data_ptr()), m, n, nq, code,
                                 ctypes.c_void_p(Q.data_ptr()), _stream(stream)))
    return Q.t()


def qtt_debug_set_tc_gemm(on):
    """Select the large-rank rounding's product kernel: tensor cores (True)
    or the CUDA-core compensated GEMM (False, the default)."""
    load()
    _lib.qtt_debug_set_tc_gemm(int(on) if on in (0, 1, 2) else int(bool(on)))


def qtt_from_cores(cores, shape_log2, interleave=True, stream=None):
    """Handle from host cores (numpy arrays (r_{k-1}, 2, r_k))."""
    load()
    d = len(cores)
    code = QTT_F64 if cores[0].dtype == np.float64 else QTT_C64
    nd = _np_dtype(code)
    ranks = [1] + [int(c.shape[2]) for c in cores]
    buf = np.concatenate([np.asarray(c, dtype=nd).reshape(-1, order="F") for c in cores])
    buf = np.ascontiguousarray(buf)
    r = (ctypes.c_int * (d + 1))(*ranks)
    sh = (ctypes.c_int * 2)(*(list(shape_log2) + [0] * (2 - len(shape_log2))))
    out = ctypes.c_void_p()
    _check(_lib.qtt_from_cores(buf.ctypes.data_as(ctypes.c_void_p), r, d, code, len(shape_log2),
                               sh, int(interleave), _stream(stream), ctypes.byref(out)))
    return QTTTensor(out)


def _line_arrays(xs, ys):
    if len(xs) != len(ys):
        raise ValueError("xs and ys differ in length")
    code = _dtype_code(xs[0])
    lg = []
    for x, y in zip(xs, ys):
        if (not x.is_cuda or not y.is_cuda or not x.is_contiguous() or not y.is_contiguous()
                or x.dim() != 1 or x.shape != y.shape or x.dtype != y.dtype or _dtype_code(x) != code):
            raise ValueError("lines must be contiguous 1D CUDA tensors of one dtype, y like x")
        n = int(x.shape[0])
        ln = n.bit_length() - 1
        if n < 4 or (1 << ln) != n:
            raise ValueError(f"line length {n} is not a power of two >= 4")
        lg.append(ln)
    xp = (ctypes.c_void_p * len(xs))(*[x.data_ptr() for x in xs])
    yp = (ctypes.c_void_p * len(ys))(*[y.data_ptr() for y in ys])
    return code, lg, xp, yp


class QTTBatch:
    """Independent 1D lines of uneven length, bandwidth and rank cap through
    decompose -> sinc convolution -> Full, spread over ``nstreams`` internal
    streams; ``capture`` records the whole batch as one CUDA graph that
    ``launch`` replays."""

    def __init__(self, log2_len, B, rmax, eps=0.0, refine=True, normalize=True, eps_op=1e-7,
                 eps_round=1e-7, rround=0, dtype_code=QTT_C64, nstreams=0, stream=None):
        load()
        n = len(log2_len)
        self.n = n
        self.log2_len = [int(v) for v in log2_len]
        tr = _trunc(eps_round, rround, True)
        out = ctypes.c_void_p()
        _check(_lib.qtt_batch_create(n, (ctypes.c_int * n)(*self.log2_len),
                                     (ctypes.c_double * n)(*[float(b) for b in B]),
                                     (ctypes.c_int * n)(*[int(r) for r in rmax]), float(eps),
                                     int(bool(refine)), int(bool(normalize)), float(eps_op),
                                     ctypes.byref(tr), int(dtype_code), int(nstreams),
                                     _stream(stream), ctypes.byref(out)))
        self._h = out
        self._bufs = None
        self.tiles = (0, 0)

    def run(self, xs, ys, stream=None):
        _, lg, xp, yp = _line_arrays(xs, ys)
        if lg != self.log2_len:
            raise ValueError("line lengths differ from the batch plan")
        _check(_lib.qtt_batch_run(self._h, xp, yp, _stream(stream)))
        return ys

    def capture(self, xs, ys, stream):
        _, lg, xp, yp = _line_arrays(xs, ys)
        if lg != self.log2_len:
            raise ValueError("line lengths differ from the batch plan")
        _check(_lib.qtt_batch_capture(self._h, xp, yp, _stream(stream)))
        self._bufs = (xs, ys)      # the graph reads and writes these buffers

    def launch(self, stream=None):
        _check(_lib.qtt_batch_launch(self._h, _stream(stream)))

    def set_tiles(self, gram_parts_per_sm=0, chunk_div=0):
        """Tile settings of the lines' Gram passes (0: defaults); drops a
        captured graph."""
        f = _lib.qtt_batch_set_tiles
        f.restype = ctypes.c_int
        f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
        _check(f(self._h, int(gram_parts_per_sm), int(chunk_div)))
        self.tiles = (int(gram_parts_per_sm), int(chunk_div))

    def info(self):
        ns, nn = ctypes.c_int(), ctypes.c_int()
        _check(_lib.qtt_batch_info(self._h, ctypes.byref(ns), ctypes.byref(nn)))
        return {"nstreams": ns.value, "graph_nodes": nn.value}

    def free(self):
        if self._h is not None and self._h.value:
            _lib.qtt_batch_free(self._h)
        self._h = None
        self._bufs = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def qtt_batch_conv_sinc(xs, B, rmax, ys=None, eps=0.0, refine=True, normalize=True, eps_op=1e-7,
                        eps_round=1e-7, rround=0, stream=None):
    """One-shot batched decompose -> convolve -> Full of the 1D lines xs."""
    import torch
    load()
    if ys is None:
        ys = [torch.empty_like(x) for x in xs]
    code, lg, xp, yp = _line_arrays(xs, ys)
    n = len(xs)
    tr = _trunc(eps_round, rround, True)
    _check(_lib.qtt_batch_conv_sinc(n, xp, (ctypes.c_int * n)(*lg),
                                    (ctypes.c_double * n)(*[float(b) for b in B]),
                                    (ctypes.c_int * n)(*[int(r) for r in rmax]), float(eps),
                                    int(bool(refine)), int(bool(normalize)), float(eps_op),
                                    ctypes.byref(tr), yp, code, _stream(stream)))
    return ys


def autotune_batch(xs, ys, B, rmax, candidates=(8, 16, 32, 64), reps=2, stream=None,
                   tiles=((0, 0),), **kw):
    """Pick the internal stream count and the Gram passes' tile settings
    (``tiles``: (gram_parts_per_sm, chunk_div) pairs, (0, 0) = the defaults)
    of a captured batch by timing graph launches (CUDA events on ``stream``).
    Streams are searched first with the default tiles, then the tiles with
    the best stream count.  Returns (best QTTBatch, {(S, parts, div): ms})."""
    import torch
    if stream is None:
        stream = torch.cuda.Stream()
    lg = [int(x.shape[0]).bit_length() - 1 for x in xs]
    state = {"best": None, "ms": None}
    times = {}

    def trial(S, t):
        b = QTTBatch(lg, B, rmax, nstreams=S, stream=stream, **kw)
        if t != (0, 0):
            b.set_tiles(*t)
        b.capture(xs, ys, stream)
        b.launch(stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            b.launch(stream)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        times[(b.info()["nstreams"],) + tuple(t)] = ms
        if state["best"] is None or ms < state["ms"]:
            if state["best"] is not None:
                state["best"].free()
            state["best"], state["ms"] = b, ms
        else:
            b.free()

    for S in candidates:
        if S > len(xs) and times:
            continue
        trial(S, (0, 0))
    S_best = state["best"].info()["nstreams"]
    for t in tiles:
        if tuple(t) != (0, 0):
            trial(S_best, tuple(t))
    return state["best"], times


def qtt_small_eigh(G, dtype_code=QTT_C64, stream=None):
    """Eigen-decomposition of a small Hermitian matrix with the library's
    one-CTA solver: G (n x n, numpy or CUDA tensor) -> (lam desc, U)."""
    import torch
    load()
    G = np.asarray(G.cpu().numpy() if hasattr(G, "cpu") else G, dtype=np.complex128)
    n = G.shape[0]
    Gd = torch.from_numpy(np.ascontiguousarray(G.T)).cuda()       # column-major
    dt = torch.float64 if dtype_code == QTT_F64 else torch.complex64
    U = torch.empty((n, n), dtype=dt, device="cuda")
    lam = torch.empty(n, dtype=torch.float64, device="cuda")
    _check(_lib.qtt_small_eigh(ctypes.c_void_p(Gd.data_ptr()), n, int(dtype_code),
                               ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(lam.data_ptr()),
                               _stream(stream)))
    return lam.cpu().numpy(), U.cpu().numpy().T.copy()            # U[:, c] = eigenvector c


def qtt_debug_set_eig_solver(which):
    load()
    _lib.qtt_debug_set_eig_solver(int(which))


def version():
    load()
    return _lib.qtt_version().decode()
