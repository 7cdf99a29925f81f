"""Differentiation of the convolution step on the GPU: inner products, TT
sums, the adjoint operator, core gradients (against the oracle's dense
adjoint and against central finite differences) and gradient descent."""
import numpy as np
import pytest

from oracle import qtt as Q, conv as C, pipeline as P
from synth import scenes as S

pytestmark = pytest.mark.gpu

B1 = 24.0


def _rand_cores(rng, d, r, cplx):
    ranks = [1] + [min(r, 2 ** k, 2 ** (d - k)) for k in range(1, d)] + [1]
    out = []
    for k in range(d):
        c = rng.standard_normal((ranks[k], 2, ranks[k + 1]))
        if cplx:
            c = c + 1j * rng.standard_normal(c.shape)
        out.append(c / np.sqrt(2 * ranks[k]))
    return out


def _handle(q, cores, shape_log2):
    return q.qtt_from_cores(cores, shape_log2)


def _dense(cores, shape):
    return P.to_array(cores, shape)


def _qtt_order(w, shape):
    return w.reshape(-1) if len(shape) == 1 else Q.image_to_qtt_vector(w)


CASES = [((1024,), False), ((1024,), True), ((32, 32), False), ((32, 32), True)]


def _tol(cplx, fp64, fp32):
    return fp32 if cplx else fp64


@pytest.mark.parametrize("shape,cplx", CASES)
def test_dot_and_add_match_dense(qlib, shape, cplx):
    q = qlib
    rng = np.random.default_rng(11)
    lg = [int(np.log2(n)) for n in shape]
    d = sum(lg)
    cx, cy = _rand_cores(rng, d, 6, cplx), _rand_cores(rng, d, 5, cplx)
    if cplx:
        cx = [c.astype(np.complex64).astype(np.complex128) for c in cx]
        cy = [c.astype(np.complex64).astype(np.complex128) for c in cy]
    x, y = _handle(q, cx, lg), _handle(q, cy, lg)
    fx, fy = _dense(cx, shape), _dense(cy, shape)
    ref = np.vdot(fx, fy)
    got = q.qtt_dot(x, y).cpu().numpy()
    scale = np.linalg.norm(fx) * np.linalg.norm(fy)
    assert abs(complex(got[0], got[1]) - ref) <= _tol(cplx, 1e-13, 1e-6) * scale
    z = q.qtt_add(0.5, x, -2.0, y)
    assert z.ranks()[1:-1] == [a + b for a, b in zip(x.ranks()[1:-1], y.ranks()[1:-1])]
    fz = q.qtt_to_full(z).cpu().numpy()
    want = 0.5 * fx - 2.0 * fy
    assert C.rel_l2(fz, want) <= _tol(cplx, 1e-13, 1e-6)


@pytest.mark.parametrize("shape,cplx", CASES)
def test_adjoint_matches_dense_and_identity(qlib, shape, cplx):
    """round(T^H r) against the oracle's dense T^H (= T for the even sinc),
    and <T x, y> = <x, T^H y> through the library alone."""
    q = qlib
    rng = np.random.default_rng(12)
    lg = [int(np.log2(n)) for n in shape]
    d = sum(lg)
    eps = 1e-7 if cplx else 1e-12
    cr = _rand_cores(rng, d, 4, cplx)
    r = _handle(q, cr, lg)
    adj = q.qtt_conv_adjoint(None, r, B1, eps_op=eps, eps_round=eps)
    got = q.qtt_to_full(adj).cpu().numpy()
    ref = P.conv_dense(_dense(cr, shape), B1)
    assert C.rel_l2(got, ref) <= _tol(cplx, 1e-10, 2e-5)
    cx = _rand_cores(rng, d, 3, cplx)
    x = _handle(q, cx, lg)
    tx = q.qtt_conv_sinc(x, B1, eps_op=eps, eps_round=eps)
    lhs = q.qtt_dot(tx, r).cpu().numpy()
    rhs = q.qtt_dot(x, adj).cpu().numpy()
    scale = np.linalg.norm(_dense(cx, shape)) * np.linalg.norm(_dense(cr, shape))
    assert abs(complex(*lhs) - complex(*rhs)) <= _tol(cplx, 1e-10, 1e-5) * scale


def _problem_data(q, shape, cplx, seed=13, rank_g=8):
    """Target g (QTT of a blurred scene + noise) and a start f (rank 4)."""
    import torch
    rng = np.random.default_rng(seed)
    if len(shape) == 1:
        if cplx:
            _, scene = S.line_1d_scatterers(rng, shape[0], nscat=6, nbumps=2, bump_w=0.05)
        else:
            _, scene = S.line_1d_bumps(rng, shape[0], nbumps=4)
    else:
        scene = S.deconv_scene_2d(rng, shape[0], shape[1], nscat=6)
        if not cplx:
            scene = scene.real
    gd = P.conv_dense(scene, B1)
    gd = gd + 0.01 * np.linalg.norm(gd) / np.sqrt(gd.size) * rng.standard_normal(gd.shape)
    dt = torch.complex64 if cplx else torch.float64
    gt = torch.from_numpy(np.ascontiguousarray(gd)).to(device="cuda", dtype=dt)
    g = q.qtt_decompose(gt, eps=0.0, rmax=rank_g, refine=True)
    f0 = q.qtt_decompose(gt, eps=0.0, rmax=4, refine=True)
    return g, f0


@pytest.mark.parametrize("shape,cplx", CASES)
def test_core_grads_match_oracle_dense_adjoint(qlib, shape, cplx):
    """GPU core gradients of ||T full(F) - g||^2 against the oracle's dense
    gradient 2 T^H (T f - g) contracted with F's partial products."""
    import torch
    from paper_2301_13339_gb300.deconv import SincDeconvProblem
    q = qlib
    eps = 1e-7 if cplx else 1e-12
    g, f0 = _problem_data(q, shape, cplx)
    prob = SincDeconvProblem(g, B1, eps_op=eps, eps_round=eps)
    cores = [c.requires_grad_(True) for c in q.core_tensors(f0)]
    L = prob.loss(cores)
    grads = torch.autograd.grad(L, cores)
    cf = [c.detach().cpu().numpy().astype(np.complex128 if cplx else np.float64) for c in cores]
    gq = [c.astype(np.complex128 if cplx else np.float64) for c in g.cores()]
    gdense = _dense(gq, shape)
    w = P.deconv_dense_grad(cf, shape, B1, gdense)
    ref = P.core_grads(cf, _qtt_order(w, shape))
    Lref = P.deconv_loss(cf, shape, B1, gdense)
    assert abs(L.item() - Lref) <= _tol(cplx, 1e-9, 1e-4) * max(Lref, 1e-30) + _tol(cplx, 0, 1e-6) * np.linalg.norm(gdense) ** 2
    num = np.sqrt(sum(np.linalg.norm(gk.cpu().numpy() - rk) ** 2 for gk, rk in zip(grads, ref)))
    den = np.sqrt(sum(np.linalg.norm(rk) ** 2 for rk in ref))
    # The gradient is linear in the residual r = T f - g, which the GPU forms
    # as a difference of two rounded QTT tensors: each rounding is accurate to
    # u relative to its own norm (u = eps_round on the FP64 path; 2e-6 on the
    # FP32 path, the accuracy its roundings reach against the FP64 oracle),
    # so |dr| <= u (||T f|| + ||g||) and the adjoint's rounding adds u ||r||:
    # |d grad| / |grad| <= u (1 + kappa), kappa = (||T f|| + ||g||) / ||r||.
    Tf = P.conv_dense(_dense(cf, shape), B1)
    kappa = (np.linalg.norm(Tf) + np.linalg.norm(gdense)) / np.sqrt(Lref)
    u = _tol(cplx, 1e-12, 2e-6)
    bound = 3.0 * u * (1.0 + kappa)
    assert bound <= _tol(cplx, 1e-8, 2e-3)
    assert num <= bound * den, f"gradient error {num / den:.2e} > {bound:.2e} (kappa {kappa:.1f})"


@pytest.mark.parametrize("shape", [(1024,), (32, 32)])
def test_core_grads_central_differences_fp64(qlib, shape):
    """Central differences (h = 1e-3, FP64) on 24 random core entries.  The
    loss is quadratic in any single core entry, so the central difference is
    exact up to rounding."""
    import torch
    from paper_2301_13339_gb300.deconv import SincDeconvProblem
    q = qlib
    g, f0 = _problem_data(q, shape, False, seed=21)
    prob = SincDeconvProblem(g, B1, eps_op=1e-12, eps_round=1e-12)
    cores = [c.requires_grad_(True) for c in q.core_tensors(f0)]
    L = prob.loss(cores)
    grads = [gk.cpu().numpy() for gk in torch.autograd.grad(L, cores)]
    gmax = max(np.abs(gk).max() for gk in grads)
    rng = np.random.default_rng(5)
    h = 1e-3
    checked = 0
    with torch.no_grad():
        base = [c.detach().clone() for c in cores]
        while checked < 24:
            k = int(rng.integers(0, len(base)))
            idx = tuple(int(rng.integers(0, s)) for s in base[k].shape)
            vals = []
            for sgn in (1.0, -1.0):
                cs = [c.clone() for c in base]
                cs[k][idx] += sgn * h
                vals.append(prob.loss(cs).item())
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - grads[k][idx]) <= 1e-6 * gmax + 1e-6 * abs(fd), (k, idx, fd, grads[k][idx])
            checked += 1


@pytest.mark.parametrize("cplx", [False, True])
def test_recomputed_residual_gives_identical_gradient(qlib, cplx):
    import torch
    from paper_2301_13339_gb300.deconv import SincDeconvProblem
    q = qlib
    g, f0 = _problem_data(q, (1024,), cplx, seed=22)
    eps = 1e-7 if cplx else 1e-12
    out = []
    for budget in (256 << 20, 0):
        prob = SincDeconvProblem(g, B1, eps_op=eps, eps_round=eps, store_budget_bytes=budget)
        cores = [c.requires_grad_(True) for c in q.core_tensors(f0)]
        out.append([gk.cpu().numpy() for gk in torch.autograd.grad(prob.loss(cores), cores)])
        assert prob.recomputed == (1 if budget == 0 else 0)
    for a, b in zip(*out):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("shape,cplx", CASES)
def test_gradient_descent_decreases_loss(qlib, shape, cplx):
    from paper_2301_13339_gb300.deconv import (SincDeconvProblem, deconvolve,
                                                lipschitz_estimate, default_step)
    q = qlib
    g, f0 = _problem_data(q, shape, cplx, seed=23)
    eps = 1e-7 if cplx else 1e-12
    prob = SincDeconvProblem(g, B1, eps_op=eps, eps_round=eps)
    L_hat = lipschitz_estimate(prob)
    assert 0.5 < L_hat < 4.0          # 2 ||T||^2 for the unit-mass sinc kernel
    cores0 = q.core_tensors(f0)
    _, losses = deconvolve(prob, cores0, 20, default_step(prob, cores0, L_hat))
    L = losses.cpu().numpy()
    gn2 = float(q.qtt_dot(g, g)[0].item())
    slack = (1e-6 if cplx else 1e-12) * gn2      # rounding noise of the loss
    assert np.all(np.diff(L) <= slack), L
    assert L[-1] < L[0]
