"""Gradients of a least-squares loss through the SIPG solve (differentiation
of the discrete problem of Sec. 2, Eq. mat_form; the paper has no adjoint).

Test infrastructure only (see ``oracle/__init__.py``).

Problem: A(kappa, gamma) u = b(f) = M_h f, where A = kappa (A_c + gamma A_p) on
a uniform mesh, gamma the face penalty value of every face of the finest
level and A_p the penalty-only form with unit penalty (``assembly.assemble``
with part="penalty" and kappa = 1).  Loss J = 1/2 ||u - u_obs||_2^2 over DoF
vectors.  With lambda = A^{-T} (u - u_obs) = A^{-1} (u - u_obs) (A symmetric):
  dJ/df     = M_h^T lambda = M_h lambda
  dJ/dkappa = -lambda^T (dA/dkappa) u = -lambda^T A u / kappa = -lambda^T b / kappa
  dJ/dgamma = -lambda^T (dA/dgamma) u = -kappa lambda^T A_p u
"""
import numpy as np

from .assembly import assemble, block_apply, element_blocks, mass_apply, penalty
from .direct import GlobalFD


def eta_from_gamma(k, N, gamma):
    """Penalty multiplier eta such that gamma_e = gamma on every face."""
    return gamma / penalty(k, N, 1.0)


def forward(dim, k, N, f, kappa, gamma):
    """u = A^{-1} M_h f, exact (global fast diagonalisation)."""
    eta = eta_from_gamma(k, N, gamma)
    fd = GlobalFD(dim, k, N, kappa, eta)
    b = mass_apply(dim, k, N, f)
    return fd.solve(b), b, fd


def loss_and_gradients(dim, k, N, f, kappa, gamma, u_obs):
    u, b, fd = forward(dim, k, N, f, kappa, gamma)
    res = u - u_obs
    J = 0.5 * res @ res
    lam = fd.solve(res)
    Ap = assemble(dim, k, N, 1.0, 1.0, part="penalty")
    g_f = mass_apply(dim, k, N, lam)
    g_kappa = -(lam @ b) / kappa
    g_gamma = -kappa * (lam @ (Ap @ u))
    return J, g_f, g_kappa, g_gamma, u, lam


def loss_and_gradients_blocks(dim, k, N, f, kappa, gamma, u_obs):
    """Same as ``loss_and_gradients`` with A_p u evaluated cell by cell from the
    element blocks (no assembled matrix), for meshes too large to assemble."""
    u, b, fd = forward(dim, k, N, f, kappa, gamma)
    res = u - u_obs
    J = 0.5 * res @ res
    lam = fd.solve(res)
    Apu = block_apply(dim, k, N, element_blocks(dim, k, N, 1.0, 1.0, part="penalty"), u).ravel()
    g_f = mass_apply(dim, k, N, lam)
    g_kappa = -(lam @ b) / kappa
    g_gamma = -kappa * (lam @ Apu)
    return J, g_f, g_kappa, g_gamma, u, lam
