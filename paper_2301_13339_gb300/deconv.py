"""Gradient-based deconvolution in QTT form.

Loss of a QTT tensor F (cores F_1 .. F_d) against a target g held in QTT
form (typically the TT-SVD of the observed, sinc-blurred data, Alg. 1):

    L(F) = || T full(F) - g ||^2

with T the sinc Toeplitz operator of ``qtt_conv_sinc`` (Eq. GAF).  The
forward pass forms the residual r = round(round(T F) - g) and its squared
norm <r, r>; the backward pass is the library's adjoint kernel:
w = 2 round(T^H r) contracted with the partial products of F's cores
(``qtt_conv_adjoint``).  Every step runs in libqtt; PyTorch holds the core
tensors and the autograd graph.

Core tensors are CUDA tensors of shape (r_{k-1}, 2, r_k) stored column-major
(``empty_cores`` / ``core_tensors`` make them), dtype float64 (FP64 path) or
complex64 (FP32 path).  For complex cores the gradient follows PyTorch's
convention for real losses of complex leaves (2 dL/d conj(F_k)).

Memory policy: the forward residual r is kept for the backward pass when its
cores fit in ``store_budget_bytes``; otherwise it is freed and recomputed from
F in the backward pass (the same seeds give the same rounding, so the
gradient is identical either way).

Large ranks (a sketch rank above QTT_RANK_CAP, the rounding's large-rank
mode): the residual is never rounded as a sum, whose rank would be that of
T F plus that of g.  The loss is ||y||^2 - 2 Re <g, y> + ||g||^2 with
y = round(T F), and the gradient is linear in the residual:
2 C(F, round(T^H y)) - 2 C(F, round(T^H g)), with round(T^H g) formed once
per target.
"""
import torch

from . import (QTT_RANK_CAP, qtt_add, qtt_conv_adjoint, qtt_conv_sinc, qtt_core_grads, qtt_dot,
               qtt_from_device_cores, qtt_round, empty_cores)

__all__ = ["SincDeconvProblem", "deconvolve", "lipschitz_estimate", "default_step"]


class SincDeconvProblem:
    """The loss L(F) = ||T full(F) - g||^2 for a fixed target g (QTTTensor).

    B, normalize, eps_op     the sinc operator (as ``qtt_conv_sinc``).
    eps_round, rround        truncation of every rounding (T F, the
                             residual, T^H r).
    store_budget_bytes       keep the residual between forward and backward
                             when its cores fit (0: always recompute).
    """

    def __init__(self, g, B, normalize=True, eps_op=1e-7, eps_round=1e-7, rround=0,
                 sketch=0, seed=20230131, store_budget_bytes=256 << 20):
        self.g = g
        self.B = B
        self.normalize = normalize
        self.eps_op = eps_op
        self.eps_round = eps_round
        self.rround = rround
        self.sketch = sketch
        self.seed = seed
        self.store_budget_bytes = store_budget_bytes
        self.shape_log2 = g.log2_shape
        self.interleave = g.interleave
        self.recomputed = 0
        self.split = sketch > QTT_RANK_CAP     # large-rank mode: no rounded residual
        self._gadj = None                      # (g, round(T^H g), <g, g>) of the split form

    def split_terms(self):
        """round(T^H g) and <g, g> for the current target (formed once)."""
        if self._gadj is None or self._gadj[0] is not self.g:
            if self._gadj is not None:
                self._gadj[1].free(torch.cuda.current_stream())
            adj = qtt_conv_adjoint(None, self.g, self.B, self.normalize, self.eps_op,
                                   self.eps_round, self.rround, True, self.sketch, self.seed + 4)
            self._gadj = (self.g, adj, qtt_dot(self.g, self.g)[0].clone())
        return self._gadj[1], self._gadj[2]

    def forward_split(self, f):
        """y = round(T f) and the loss ||y||^2 - 2 Re <g, y> + ||g||^2."""
        y = qtt_conv_sinc(f, self.B, self.normalize, self.eps_op, self.eps_round, self.rround,
                          True, self.sketch, self.seed)
        _, gg = self.split_terms()
        val = qtt_dot(y, y)[0] - 2.0 * qtt_dot(self.g, y)[0] + gg
        return y, val

    def grads_split(self, f, y, grads):
        """2 C(f, round(T^H y)) - 2 C(f, round(T^H g)) into grads."""
        wy = qtt_conv_adjoint(None, y, self.B, self.normalize, self.eps_op, self.eps_round,
                              self.rround, True, self.sketch, self.seed + 2)
        wg, _ = self.split_terms()
        qtt_core_grads(f, wy, grads, alpha=2.0, beta=0.0)
        qtt_core_grads(f, wg, grads, alpha=-2.0, beta=1.0)
        wy.free(torch.cuda.current_stream())

    # ------------------------------------------------------------ pieces
    def handle(self, cores):
        return qtt_from_device_cores([c.detach() for c in cores], self.shape_log2, self.interleave)

    def residual(self, f):
        """r = round(round(T f) - g) as a new QTTTensor."""
        y = qtt_conv_sinc(f, self.B, self.normalize, self.eps_op, self.eps_round, self.rround,
                          True, self.sketch, self.seed)
        r = qtt_add(1.0, y, -1.0, self.g)
        y.free(torch.cuda.current_stream())
        qtt_round(r, self.eps_round, self.rround, True, self.sketch, self.seed + 1)
        return r

    def grads_into(self, f, r, grads):
        qtt_conv_adjoint(f, r, self.B, self.normalize, self.eps_op, self.eps_round, self.rround,
                         True, self.sketch, self.seed + 2, grad_cores=grads, want_adj=False)

    def loss(self, cores):
        """L as a 0-dim CUDA float64 tensor, differentiable w.r.t. the cores."""
        return _SincDeconvLoss.apply(self, *cores)


class _SincDeconvLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, problem, *cores):
        f = problem.handle(cores)
        ranks = [1] + [int(c.shape[2]) for c in cores]
        if problem.split:
            y, val = problem.forward_split(f)
            ctx.problem = problem
            ctx.f = f
            ctx.r = y
            ctx.ranks = ranks
            ctx.dtype = cores[0].dtype
            return val.clone()
        r = problem.residual(f)
        val = qtt_dot(r, r)
        # upper bound of the residual's core storage (ranks <= QTT_RANK_CAP)
        rbytes = cores[0].element_size() * len(cores) * 2 * QTT_RANK_CAP * QTT_RANK_CAP
        if rbytes > problem.store_budget_bytes:
            r.free(torch.cuda.current_stream())
            r = None
        ctx.problem = problem
        ctx.f = f
        ctx.r = r
        ctx.ranks = ranks
        ctx.dtype = cores[0].dtype
        return val[0].clone()

    @staticmethod
    def backward(ctx, gout):
        problem = ctx.problem
        r = ctx.r
        grads = empty_cores(ctx.ranks, ctx.dtype)
        if problem.split:
            problem.grads_split(ctx.f, r, grads)
        else:
            if r is None:
                r = problem.residual(ctx.f)
                problem.recomputed += 1
            problem.grads_into(ctx.f, r, grads)
        stream = torch.cuda.current_stream()
        r.free(stream)
        ctx.f.free(stream)
        ctx.f = None
        ctx.r = None
        real = torch.float64 if ctx.dtype == torch.float64 else torch.float32
        s = gout.to(real)
        return (None, *[g.mul_(s) for g in grads])


def lipschitz_estimate(problem, iters=10, eps=1e-4):
    """2 lambda_max(T^H T): the Lipschitz constant of f -> 2 T^H (T f - g),
    from `iters` power iterations started at g (Rayleigh quotients; every
    product rounded at `eps`, enough for a step size)."""
    x = problem.g
    lam = 0.0
    for _ in range(iters):
        y = qtt_conv_sinc(x, problem.B, problem.normalize, problem.eps_op, eps, 0, True,
                          problem.sketch, problem.seed)
        z = qtt_conv_adjoint(None, y, problem.B, problem.normalize, problem.eps_op, eps, 0, True,
                             problem.sketch, problem.seed + 3)
        num = qtt_dot(x, z)[0]
        den = qtt_dot(x, x)[0]
        lam = float((num / den).item())
        x = z
    return 2.0 * lam


def default_step(problem, cores, L_hat=None):
    """Fixed step 0.5 / (L_hat d max(1, ||f||^2)) for plain gradient descent
    on the d cores of a TT-SVD-shaped f (cores 1..d-1 left-orthonormal, the
    norm in the last core): each core's block of the gradient is at most
    L_hat ||f||^2 Lipschitz, and all d blocks move at once."""
    if L_hat is None:
        L_hat = lipschitz_estimate(problem)
    f = problem.handle(cores)
    fn2 = float(qtt_dot(f, f)[0].item())
    return 0.5 / (L_hat * len(cores) * max(1.0, fn2))


def deconvolve(problem, cores, steps, step_size):
    """Plain gradient descent on the cores: F_k <- F_k - step_size * grad_k.
    Returns the updated cores and the loss before every step (CUDA tensor)."""
    cores = [c.detach().clone() for c in cores]      # clone keeps the column-major strides
    for c in cores:
        c.requires_grad_(True)
    losses = torch.empty(steps + 1, dtype=torch.float64, device="cuda")
    for it in range(steps):
        L = problem.loss(cores)
        losses[it] = L.detach()
        grads = torch.autograd.grad(L, cores)
        with torch.no_grad():
            for c, g in zip(cores, grads):
                c.sub_(step_size * g)
    with torch.no_grad():
        losses[steps] = problem.loss(cores)
    return [c.detach() for c in cores], losses
