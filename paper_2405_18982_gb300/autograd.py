"""Differentiable SIPG solve: u = A(kappa, gamma)^{-1} M_h f.

A = kappa (A_c + gamma A_p) is the fine-level SIPG matrix of Sec. 2 with a
uniform face penalty value gamma (gamma = 2 eta k(k+1)/h on every face of the
uniform mesh) and A_p the penalty form with unit penalty; b = M_h f for a
source given by nodal values.  The backward pass is the adjoint: A is
symmetric, so lambda = A^{-1} g is a second MG-preconditioned FCG solve on the
incoming gradient g = dJ/du, and
    dJ/df     = M_h lambda
    dJ/dkappa = -lambda^T (dA/dkappa) u = -lambda^T b / kappa
    dJ/dgamma = -lambda^T (dA/dgamma) u = -lambda^T (kappa A_p u).
Every vector operation runs in the CUDA library (sipg_rhs, sipg_solve,
sipg_adjoint_solve, sipg_apply_penalty, sipg_dot); Python only marshals.
"""
import torch

from . import SIPG, SIPG_FP32, SIPG_FP64, Params


class SolverCache:
    """SIPG handles per (kappa, eta): the level setup depends on both."""

    def __init__(self, dim, degree, log2_cells, n_levels, nrhs=1, vcycle_precision=SIPG_FP32,
                 use_graphs=1, device=None):
        self.base = dict(dim=dim, degree=degree, log2_cells=log2_cells, n_levels=n_levels, nrhs=nrhs,
                         vcycle_precision=vcycle_precision, use_graphs=use_graphs)
        self.device = device
        self._cache = {}

    def gamma_unit(self):
        """gamma of eta = 1 on the finest level: 2 k (k+1) / h."""
        k = self.base["degree"]
        return 2.0 * k * (k + 1) * (1 << self.base["log2_cells"])

    def get(self, kappa, gamma):
        eta = gamma / self.gamma_unit()
        key = (float(kappa), float(eta))
        s = self._cache.get(key)
        if s is None:
            s = SIPG(Params(kappa=float(kappa), penalty_factor=float(eta), **self.base), device=self.device)
            self._cache[key] = s
        return s


class SIPGSolveFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, kappa, gamma, cache, rtol, maxit):
        s = cache.get(float(kappa), float(gamma))
        f64 = f.detach().to(torch.float64).contiguous()
        b = torch.empty_like(f64)
        s.rhs(f64, b)
        u = torch.zeros_like(f64)
        s.solve(b, u, rtol=rtol, maxit=maxit)
        ctx.s = s
        ctx.rtol, ctx.maxit = rtol, maxit
        ctx.kappa = float(kappa)
        ctx.f_dtype = f.dtype
        ctx.k_like = (kappa.device, kappa.dtype)
        ctx.g_like = (gamma.device, gamma.dtype)
        ctx.save_for_backward(u, b)
        return u

    @staticmethod
    def backward(ctx, g):
        s = ctx.s
        u, b = ctx.saved_tensors
        g = g.to(torch.float64).contiguous()
        lam = torch.zeros_like(g)
        s.adjoint_solve(g, lam, rtol=ctx.rtol, maxit=ctx.maxit)
        grad_f = grad_k = grad_g = None
        if ctx.needs_input_grad[0]:
            gf = torch.empty_like(lam)
            s.rhs(lam, gf)                       # M_h lambda
            grad_f = gf.to(ctx.f_dtype)
        nrhs = lam.shape[0] if lam.dim() == 2 else 1
        dots = torch.zeros(nrhs, dtype=torch.float64, device=lam.device)
        if ctx.needs_input_grad[1]:
            s.dot(lam, b, dots)
            grad_k = (-dots.sum() / ctx.kappa).reshape(()).to(*ctx.k_like)
        if ctx.needs_input_grad[2]:
            apu = torch.empty_like(u)
            s.apply_penalty(u, apu)              # (dA/dgamma) u = kappa A_p u
            s.dot(lam, apu, dots)
            grad_g = (-dots.sum()).reshape(()).to(*ctx.g_like)
        return grad_f, grad_k, grad_g, None, None, None


def sipg_solve(f, kappa, gamma, cache, rtol=1e-10, maxit=200):
    """u = A(kappa, gamma)^{-1} M_h f, differentiable in f, kappa and gamma.

    f: (nrhs, ndofs) CUDA tensor (any float dtype; promoted to FP64);
    kappa, gamma: 0-dim tensors (or floats); cache: SolverCache."""
    if not torch.is_tensor(kappa):
        kappa = torch.tensor(float(kappa), dtype=torch.float64)
    if not torch.is_tensor(gamma):
        gamma = torch.tensor(float(gamma), dtype=torch.float64)
    return SIPGSolveFn.apply(f, kappa, gamma, cache, rtol, maxit)
