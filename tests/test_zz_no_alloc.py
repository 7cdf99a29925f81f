"""The allocation-free Full entry point (qtt_to_full_noalloc) against
qtt_to_full, through the C ABI.

It serves callers that must not allocate device memory after start-up
(latency-critical loops, processes whose device memory another allocator
already owns).  Two calls in a row check that the shared static scratch,
which keeps the previous call's contents, does not leak into the result.
This file is collected last so that a run stopping at its first failure has
already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _rand_cores(rng, d, r, dtype):
    ranks = [1] + [min(r, 2 ** k, 2 ** (d - k)) for k in range(1, d)] + [1]
    out = []
    for k in range(d):
        shp = (ranks[k], 2, ranks[k + 1])
        c = rng.standard_normal(shp)
        if dtype == np.complex64:
            c = c + 1j * rng.standard_normal(shp)
        out.append((c / np.sqrt(2 * ranks[k])).astype(dtype))
    return out


@pytest.mark.parametrize("dtype,shape,interleave,tol", [
    (np.complex64, [14], True, 1e-5), (np.float64, [12], True, 1e-12),
    (np.complex64, [6, 6], True, 1e-5), (np.complex64, [5, 7], False, 1e-5),
    (np.float64, [6, 6], True, 1e-12), (np.float64, [6, 5], False, 1e-12)])
def test_to_full_noalloc_matches_to_full(qlib, dtype, shape, interleave, tol):
    import torch
    rng = np.random.default_rng(17)
    d = sum(shape)
    first = None
    # the first call writes the larger rank, so a stale read of a column past
    # the second call's rank would show in the second result
    for call, r in enumerate((32, 8)):
        cores = _rand_cores(rng, d, r, dtype)
        t = qlib.qtt_from_cores(cores, shape, interleave=interleave)
        ref = qlib.qtt_to_full(t)
        out = torch.full_like(ref, float("nan"))
        qlib.qtt_to_full_noalloc(t, out)
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b)
        if first is None:
            first = b
        else:
            assert np.linalg.norm(b - first) > 0    # the second call expanded a different tensor


def test_to_full_noalloc_rejects_oversize(qlib):
    # d = 28 with rank 64 needs 32 MiB of scratch, above the 16 MiB static
    # limit: the C entry point must refuse before launching anything
    import ctypes
    import torch
    d = 28
    ranks = [1] + [min(64, 2 ** k, 2 ** (d - k)) for k in range(1, d)] + [1]
    cores = [np.zeros((ranks[k], 2, ranks[k + 1]), dtype=np.complex64) for k in range(d)]
    t = qlib.qtt_from_cores(cores, [d])
    out = torch.empty(1, dtype=torch.complex64, device="cuda")
    st = qlib.lib().qtt_to_full_noalloc(t.handle, ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == -1                                  # QTT_EINVAL
    assert b"static limit" in qlib.lib().qtt_last_error()
    # a successful call afterwards leaves no stale message behind
    small = qlib.qtt_from_cores([c[:1, :, :1] for c in cores[:4]], [4])
    out2 = torch.empty(16, dtype=torch.complex64, device="cuda")
    qlib.qtt_to_full_noalloc(small, out2)
    torch.cuda.synchronize()
    assert qlib.lib().qtt_last_error() == b""
