"""Pins of the oracle's gradients: a closed form in kappa, the definition of
the f-gradient through the direct solver, and FP64 central differences."""
import numpy as np
import pytest

from oracle.adjoint import eta_from_gamma, forward, loss_and_gradients
from oracle.assembly import assemble, mass_apply, penalty
from oracle.direct import GlobalFD
import scipy.sparse.linalg as spla


@pytest.mark.parametrize("dim,k,N", [(2, 2, 4), (3, 2, 2)])
def test_direct_solver_equals_sparse_solve(dim, k, N):
    rng = np.random.default_rng(20)
    A = assemble(dim, k, N, kappa=1.7, eta=1.3).tocsc()
    b = rng.standard_normal(A.shape[0])
    x = GlobalFD(dim, k, N, kappa=1.7, eta=1.3).solve(b)
    xs = spla.spsolve(A, b)
    assert np.abs(x - xs).max() < 1e-12 * np.abs(xs).max()


def _setup(dim, k, N, seed=21):
    rng = np.random.default_rng(seed)
    nd = N ** dim * (k + 1) ** dim
    f = rng.standard_normal(nd)
    u_obs = rng.standard_normal(nd) * 1e-2
    return f, u_obs


def test_kappa_gradient_closed_form():
    # u(kappa) = u_1 / kappa with u_1 the solution at kappa = 1, so
    # dJ/dkappa = -kappa^-2 u_1^T (u_1 / kappa - u_obs)
    dim, k, N = 2, 3, 4
    f, u_obs = _setup(dim, k, N)
    gamma = penalty(k, N, 1.0)
    kappa = 1.37
    J, gf, gk, gg, u, lam = loss_and_gradients(dim, k, N, f, kappa, gamma, u_obs)
    u1, _, _ = forward(dim, k, N, f, 1.0, gamma)
    expect = -(kappa ** -2) * (u1 @ (u1 / kappa - u_obs))
    assert abs(gk - expect) < 1e-12 * abs(expect)


def test_f_gradient_definition():
    dim, k, N = 2, 2, 4
    f, u_obs = _setup(dim, k, N, 22)
    gamma = 1.3 * penalty(k, N, 1.0)
    J, gf, gk, gg, u, lam = loss_and_gradients(dim, k, N, f, 0.9, gamma, u_obs)
    A = assemble(dim, k, N, 0.9, eta_from_gamma(k, N, gamma)).toarray()
    expect = mass_apply(dim, k, N, np.linalg.solve(A, u - u_obs))
    assert np.abs(gf - expect).max() < 1e-11 * np.abs(expect).max()


@pytest.mark.parametrize("dim,k,N", [(2, 2, 4), (3, 2, 2)])
def test_gradients_match_central_differences(dim, k, N):
    f, u_obs = _setup(dim, k, N, 23)
    kappa = 1.2
    gamma = penalty(k, N, 1.0)
    J, gf, gk, gg, u, lam = loss_and_gradients(dim, k, N, f, kappa, gamma, u_obs)

    def Jof(ff, kk, gm):
        uu, _, _ = forward(dim, k, N, ff, kk, gm)
        return 0.5 * np.sum((uu - u_obs) ** 2)

    step = 1e-6
    # kappa and gamma: relative steps of 1e-6
    dk = (Jof(f, kappa * (1 + step), gamma) - Jof(f, kappa * (1 - step), gamma)) / (2 * kappa * step)
    dg = (Jof(f, kappa, gamma * (1 + step)) - Jof(f, kappa, gamma * (1 - step))) / (2 * gamma * step)
    assert abs(dk - gk) < 1e-6 * abs(gk)
    assert abs(dg - gg) < 1e-5 * abs(gg) + 1e-14
    # f: directional derivative along a random direction
    rng = np.random.default_rng(24)
    dvec = rng.standard_normal(len(f))
    df = (Jof(f + step * dvec, kappa, gamma) - Jof(f - step * dvec, kappa, gamma)) / (2 * step)
    assert abs(df - gf @ dvec) < 1e-6 * abs(gf @ dvec)


@pytest.mark.parametrize("dim,k,N", [(2, 3, 4), (3, 2, 4)])
def test_block_gradients_equal_assembled_gradients(dim, k, N):
    # the cell-by-cell evaluation of A_p u (for large meshes) gives the same
    # gradients as the assembled penalty matrix
    from oracle.adjoint import loss_and_gradients_blocks
    f, u_obs = _setup(dim, k, N, 31)
    kappa, gamma = 1.4, penalty(k, N, 1.0)
    a = loss_and_gradients(dim, k, N, f, kappa, gamma, u_obs)
    b = loss_and_gradients_blocks(dim, k, N, f, kappa, gamma, u_obs)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and a[2] == b[2]
    assert abs(a[3] - b[3]) <= 1e-12 * abs(a[3])
