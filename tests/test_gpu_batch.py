"""Batched lines: the multi-stream submission and its CUDA-graph replay give
the same bits as the single-line calls, and sampled lines match the oracle."""
import numpy as np
import pytest

from oracle import pipeline as P, conv as C
from synth import scenes as S

pytestmark = pytest.mark.gpu


def _lines(n=10, dmin=9, dmax=12, seed=41):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        d = int(rng.integers(dmin, dmax + 1))
        B = float(rng.uniform(16.0, 2.0 ** d / 4))
        rmax = int(rng.choice([8, 16, 32, 64]))
        x, _ = S.line_1d_scatterers(rng, 2 ** d, nscat=int(rng.integers(10, 41)), nbumps=0,
                                    snr_db=15.0)
        out.append(dict(x=x.astype(np.complex64), d=d, B=B, rmax=rmax))
    return out


def _single(q, ln, i, stream):
    import torch
    x = torch.from_numpy(ln["x"]).cuda()
    f = q.qtt_decompose(x, eps=0.0, rmax=ln["rmax"], refine=True, stream=stream)
    y = q.qtt_conv_sinc(f, ln["B"], eps_op=1e-7, eps_round=1e-7, seed=20230131 + i,
                        stream=stream)
    return q.qtt_to_full(y, stream=stream)


def test_batch_eager_and_graph_equal_single_line_calls(qlib):
    import torch
    q = qlib
    lines = _lines()
    s = torch.cuda.Stream()
    xs = [torch.from_numpy(ln["x"]).cuda() for ln in lines]
    ys = [torch.zeros_like(x) for x in xs]
    with torch.cuda.stream(s):
        ref = [_single(q, ln, i, s) for i, ln in enumerate(lines)]
    torch.cuda.synchronize()
    b = q.QTTBatch([ln["d"] for ln in lines], [ln["B"] for ln in lines],
                   [ln["rmax"] for ln in lines], nstreams=4, stream=s)
    b.run(xs, ys, stream=s)
    s.synchronize()
    for r, y in zip(ref, ys):
        assert np.array_equal(r.cpu().numpy(), y.cpu().numpy())
    b.capture(xs, ys, s)
    assert b.info()["graph_nodes"] > 10 * len(lines)
    for _ in range(2):
        for y in ys:
            y.zero_()
        b.launch(s)
        s.synchronize()
        for r, y in zip(ref, ys):
            assert np.array_equal(r.cpu().numpy(), y.cpu().numpy())
    b.free()
    ys2 = q.qtt_batch_conv_sinc(xs, [ln["B"] for ln in lines], [ln["rmax"] for ln in lines],
                                stream=s)
    s.synchronize()
    for r, y in zip(ref, ys2):
        assert np.array_equal(r.cpu().numpy(), y.cpu().numpy())


def test_batch_lines_match_oracle(qlib):
    import torch
    q = qlib
    lines = _lines(n=6, dmin=10, dmax=11, seed=42)
    xs = [torch.from_numpy(ln["x"]).cuda() for ln in lines]
    ys = q.qtt_batch_conv_sinc(xs, [ln["B"] for ln in lines], [ln["rmax"] for ln in lines])
    torch.cuda.synchronize()
    for ln, y in list(zip(lines, ys))[:3]:
        ref = P.conv_sinc_qtt(ln["x"].astype(np.complex128), ln["B"], 0.0, ln["rmax"],
                              eps_op=1e-7, eps_round=1e-7)
        assert C.rel_l2(y.cpu().numpy().astype(np.complex128), ref) <= 1e-5


def test_autotune_picks_a_candidate(qlib):
    import torch
    q = qlib
    lines = _lines(n=8, dmin=9, dmax=10, seed=43)
    xs = [torch.from_numpy(ln["x"]).cuda() for ln in lines]
    ys = [torch.empty_like(x) for x in xs]
    best, times = q.autotune_batch(xs, ys, [ln["B"] for ln in lines],
                                   [ln["rmax"] for ln in lines], candidates=(2, 4, 8), reps=1,
                                   tiles=((0, 0), (1, 0), (0, 2)))
    key = (best.info()["nstreams"],) + tuple(best.tiles)
    assert key in times and len(times) >= 4
    assert times[key] == min(times.values())
    best.free()


@pytest.mark.parametrize("tiles", [(1, 2), (8, 4)])
def test_batch_tiles_match_oracle_and_replay(qlib, tiles):
    """Non-default Gram tiles (partial-Gram CTAs per SM, narrower column
    chunks) change the order of the FP32 sums only: sampled lines still match
    the oracle at 1e-5, and the captured graph replays the eager run's bits."""
    import torch
    q = qlib
    lines = _lines(n=6, dmin=10, dmax=12, seed=44)
    s = torch.cuda.Stream()
    xs = [torch.from_numpy(ln["x"]).cuda() for ln in lines]
    ys = [torch.zeros_like(x) for x in xs]
    b = q.QTTBatch([ln["d"] for ln in lines], [ln["B"] for ln in lines],
                   [ln["rmax"] for ln in lines], nstreams=3, stream=s)
    b.set_tiles(*tiles)
    b.run(xs, ys, stream=s)
    s.synchronize()
    eager = [y.cpu().numpy() for y in ys]
    for ln, y in list(zip(lines, eager))[:3]:
        ref = P.conv_sinc_qtt(ln["x"].astype(np.complex128), ln["B"], 0.0, ln["rmax"],
                              eps_op=1e-7, eps_round=1e-7)
        assert C.rel_l2(y.astype(np.complex128), ref) <= 1e-5
    b.capture(xs, ys, s)
    for y in ys:
        y.zero_()
    b.launch(s)
    s.synchronize()
    for e, y in zip(eager, ys):
        assert np.array_equal(e, y.cpu().numpy())
    with pytest.raises(q.QTTError):
        b.set_tiles(17, 0)
    with pytest.raises(q.QTTError):
        b.set_tiles(0, 3)
    b.free()
