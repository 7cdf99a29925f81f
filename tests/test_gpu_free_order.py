"""qtt_free releases a handle's storage in stream order after the last call
that used it (the handle's last-use event), without synchronising the
device: a Full enqueued just before the free still reads intact cores, also
when the memory pool hands the storage out again right away on another
stream."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_free_after_enqueued_full_is_ordered(qlib):
    import torch
    rng = synth.config_rng(1, sub=21)
    x, _ = synth.line_1d_scatterers(rng, 2 ** 18, nscat=40, snr_db=20.0)
    xd = torch.from_numpy(x.astype(np.complex64)).cuda()
    ref = qlib.qtt_to_full(qlib.qtt_decompose(xd, rmax=32, refine=True)).cpu().numpy()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = []
    for _ in range(4):
        with torch.cuda.stream(s1):
            f = qlib.qtt_decompose(xd, rmax=32, refine=True, stream=s1)
            out = torch.empty_like(xd)
            qlib.qtt_to_full(f, out=out, stream=s1)
            f.free()                      # qtt_free: no stream, no device synchronisation
        with torch.cuda.stream(s2):       # reuse the pool at once elsewhere
            g = qlib.qtt_decompose(torch.flip(xd, [0]), rmax=32, refine=True, stream=s2)
            junk = torch.empty_like(xd)
            qlib.qtt_to_full(g, out=junk, stream=s2)
            g.free(stream=s2)
        outs.append(out)
    torch.cuda.synchronize()
    for out in outs:
        assert np.array_equal(out.cpu().numpy(), ref)
