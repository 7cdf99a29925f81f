"""Max rank TT-RSVD (Sec. 5 modification (2), App. A Algs. 4-5) through the
C ABI against the oracle's tt_rsvd on the same Gaussian test matrices:
ranks equal, reconstruction within 1e-11 (FP64) / 1e-5 (FP32); the device
draws (omega = NULL) give a decomposition as good as the oracle's with its
own draws, reproducible per seed."""
import numpy as np
import pytest

from oracle import qtt as Q, rsvd as RS
import synth

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_fp64_parity_smooth_line(qlib):
    d, rmax, p = 12, 12, 6
    _, x = synth.line_1d_bumps(synth.config_rng(0), 2 ** d)
    flat, omega = synth.rsvd_omega_blocks(d, rmax, p, np.random.default_rng(31))
    cores, ranks, used = RS.tt_rsvd(x, d, rmax, p, omega)
    assert any(used)
    t = qlib.qtt_decompose_rsvd(_dev(x), rmax, p, omega=_dev(flat))
    assert t.ranks() == ranks
    got = qlib.qtt_to_full(t).cpu().numpy()
    ref = Q.full(cores)
    assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("d,rmax,p", [(14, 16, 8), (16, 32, 10)])
def test_c64_parity_noisy_line(qlib, d, rmax, p):
    x, _ = synth.line_1d_scatterers(synth.config_rng(1), 2 ** d, nscat=30, snr_db=20.0)
    x = x.astype(np.complex64)
    flat, omega = synth.rsvd_omega_blocks(d, rmax, p, np.random.default_rng(32), np.float32)
    cores, ranks, used = RS.tt_rsvd(x.astype(np.complex128), d, rmax, p, omega)
    assert any(used)
    t = qlib.qtt_decompose_rsvd(_dev(x), rmax, p, omega=_dev(flat))
    assert t.ranks() == ranks
    got = qlib.qtt_to_full(t).cpu().numpy().astype(np.complex128)
    ref = Q.full(cores)
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


def test_device_draws(qlib):
    d, rmax, p = 14, 16, 8
    x, _ = synth.line_1d_scatterers(synth.config_rng(1), 2 ** d, nscat=30, snr_db=20.0)
    xd = _dev(x.astype(np.complex64))
    a = qlib.qtt_to_full(qlib.qtt_decompose_rsvd(xd, rmax, p, seed=7)).cpu().numpy()
    b = qlib.qtt_to_full(qlib.qtt_decompose_rsvd(xd, rmax, p, seed=7)).cpu().numpy()
    c = qlib.qtt_to_full(qlib.qtt_decompose_rsvd(xd, rmax, p, seed=8)).cpu().numpy()
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    x128 = x.astype(np.complex128)
    ref, _, _ = Q.tt_svd(x128, d, 0.0, rmax)
    e_svd = np.linalg.norm(Q.full(ref) - x128)
    for got in (a, c):
        e = np.linalg.norm(got.astype(np.complex128) - x128)
        assert e <= 1.5 * e_svd


def test_low_qtt_rank_is_exact(qlib):
    rng = np.random.default_rng(5)
    d, r, rmax, p = 14, 3, 8, 4
    ranks = [1] + [min(r, 2 ** k, 2 ** (d - k)) for k in range(1, d)] + [1]
    cores = [(rng.standard_normal((ranks[k], 2, ranks[k + 1]))
              + 1j * rng.standard_normal((ranks[k], 2, ranks[k + 1]))) for k in range(d)]
    x = Q.full(cores)
    t = qlib.qtt_decompose_rsvd(_dev(x.astype(np.complex64)), rmax, p)
    got = qlib.qtt_to_full(t).cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - x) <= 1e-5 * np.linalg.norm(x)


def test_rsvd_argument_errors(qlib):
    import torch
    x = torch.zeros(2 ** 10, dtype=torch.complex64, device="cuda")
    with pytest.raises(qlib.QTTError):
        qlib.qtt_decompose_rsvd(x, 0, 4)
    with pytest.raises(qlib.QTTError):
        qlib.qtt_decompose_rsvd(x, 64, 40)
    with pytest.raises(ValueError):
        qlib.qtt_decompose_rsvd(x, 8, 4, omega=torch.zeros(10, device="cuda"))
    torch.cuda.synchronize()
