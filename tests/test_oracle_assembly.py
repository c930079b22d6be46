"""Pins of the oracle's SIPG assembly (Sec. 2) against a hand-worked matrix,
the mathematics of the method (symmetry, definiteness, consistency,
convergence order) and the independent Kronecker construction (Sec. 2.2)."""
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.assembly import (assemble, block_apply, cell_matrices, element_blocks,
                             l2_error, penalty, rhs_from_nodal, rhs_quadrature)
from oracle.basis import gauss_lobatto
from oracle.direct import GlobalFD, kron_sum, one_d_matrices
from oracle.layout import cellwise_to_lex, node_coordinates

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_hand_worked_1d_matrix():
    ref = np.loadtxt(os.path.join(GOLDEN, "sipg_1d_k1_N2.txt"))
    A = assemble(1, 1, 2).toarray()
    assert np.array_equal(A, ref)


def test_cell_matrices_q1_closed_form():
    K, M = cell_matrices(1, 1, 4)
    h = 0.25
    assert np.allclose(K, np.array([[1, -1], [-1, 1]]) / h, atol=1e-14)
    assert np.allclose(M, h * np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]]), atol=1e-15)


@pytest.mark.parametrize("dim,k,N", [(1, 3, 4), (2, 1, 4), (2, 2, 4), (2, 3, 2), (3, 1, 2), (3, 2, 2), (3, 2, 4)])
def test_symmetric_positive_definite(dim, k, N):
    A = assemble(dim, k, N).toarray()
    assert np.max(np.abs(A - A.T)) <= 1e-14 * np.max(np.abs(A))
    assert np.linalg.eigvalsh(A).min() > 0


@pytest.mark.parametrize("dim,k,N", [(1, 2, 4), (1, 5, 3), (2, 2, 4), (2, 4, 2), (3, 2, 2), (3, 3, 2)])
def test_consistency_reproduces_quadratic_solution(dim, k, N):
    # u = prod x_e (1 - x_e) lies in V_h for k >= 2; SIPG is consistent, so
    # the discrete solution is u itself (Galerkin orthogonality).
    def u(p):
        return np.prod(p * (1 - p), axis=1)

    def f(p):
        tot = np.zeros(len(p))
        for e in range(dim):
            others = np.prod(np.delete(p * (1 - p), e, axis=1), axis=1) if dim > 1 else 1.0
            tot += 2.0 * others
        return tot

    A = assemble(dim, k, N).tocsc()
    b = rhs_quadrature(dim, k, N, f)
    x = spla.spsolve(A, b)
    X = node_coordinates(dim, N, gauss_lobatto(k)[0])
    assert np.max(np.abs(x - u(X))) < 1e-12


@pytest.mark.parametrize("dim,k,N", [(2, 2, 4), (3, 2, 2), (2, 3, 4), (3, 1, 4)])
def test_kronecker_identity(dim, k, N):
    # Sec. 2.2: A = sum_e M (x) .. L (slot e) .. (x) M in global lexicographic order
    A = assemble(dim, k, N, kappa=1.3, eta=0.9).toarray()
    L, M = one_d_matrices(k, N, kappa=1.3, eta=0.9)
    p = cellwise_to_lex(dim, N, k + 1)
    K = kron_sum(dim, L, M)
    assert np.max(np.abs(A[np.ix_(p, p)] - K)) <= 1e-13 * np.max(np.abs(K))


def test_penalty_part_is_gamma_derivative():
    dim, k, N = 2, 3, 4
    g = penalty(k, N, 1.0)
    A1 = assemble(dim, k, N, kappa=1.0, eta=1.0).toarray()
    A2 = assemble(dim, k, N, kappa=1.0, eta=1.5).toarray()
    Ap = assemble(dim, k, N, kappa=1.0, part="penalty").toarray()
    assert np.allclose(A2 - A1, 0.5 * g * Ap, atol=1e-11 * np.abs(A1).max())
    # unit-penalty jump form is positive semidefinite with the constant... not in kernel
    # (boundary faces penalise constants): check PSD only
    assert np.linalg.eigvalsh(Ap).min() > -1e-12


def test_penalty_values():
    # gamma_e = k(k+1)(1/h^+ + 1/h^-) (Sec. 2.1)
    assert penalty(3, 8, 1.0) == 3 * 4 * 16
    assert penalty(2, 16, 2.0) == 2 * 2 * 3 * 32


@pytest.mark.parametrize("dim,k,N", [(2, 2, 4), (3, 2, 3), (3, 3, 2)])
def test_block_apply_equals_sparse_matrix(dim, k, N):
    rng = np.random.default_rng(1)
    A = assemble(dim, k, N, kappa=0.7)
    x = rng.standard_normal(A.shape[0])
    blocks = element_blocks(dim, k, N, kappa=0.7)
    y = block_apply(dim, k, N, blocks, x).ravel()
    assert np.allclose(y, A @ x, rtol=0, atol=1e-12 * np.abs(A @ x).max())
    sel = np.array([0, N ** dim - 1, N // 2])
    ys = block_apply(dim, k, N, blocks, x, sel)
    n = (k + 1) ** dim
    assert np.allclose(ys, (A @ x).reshape(-1, n)[sel], atol=1e-12 * np.abs(A @ x).max())


@pytest.mark.parametrize("dim,k,N", [(2, 2, 5), (3, 2, 4)])
def test_principal_block_equals_assembled_submatrix(dim, k, N):
    from oracle.assembly import principal_block
    from oracle.layout import dof_index
    A = assemble(dim, k, N, kappa=1.3).toarray()
    blocks = element_blocks(dim, k, N, kappa=1.3)
    n = k + 1
    rng = np.random.default_rng(2)
    for cells in ([0, 1, N, N + 1], list(rng.choice(N ** dim, size=6, replace=False)), [N ** dim - 1]):
        D = np.concatenate([np.arange(n ** dim) + c * n ** dim for c in cells])
        # same entries up to the summation order of the face contributions
        sub = A[np.ix_(D, D)]
        assert np.max(np.abs(principal_block(dim, k, N, blocks, cells) - sub)) <= 1e-14 * np.abs(A).max()


@pytest.mark.parametrize("dim,k,N", [(1, 3, 5), (2, 2, 4), (3, 2, 2)])
def test_rhs_partition_of_unity(dim, k, N):
    # sum_I int f phi_I = int f for f = 1: the total mass is 1
    b = rhs_from_nodal(dim, k, N, np.ones(N ** dim * (k + 1) ** dim))
    assert abs(b.sum() - 1.0) < 1e-13
    bq = rhs_quadrature(dim, k, N, lambda p: np.ones(len(p)))
    assert np.allclose(b, bq, atol=1e-15)


@pytest.mark.parametrize("dim,k,Ns", [(2, 1, (4, 8, 16)), (2, 2, (4, 8, 16)), (2, 3, (4, 8, 16)),
                                      (3, 1, (2, 4, 8)), (3, 2, (2, 4, 8))])
def test_manufactured_convergence_rates(dim, k, Ns):
    # u = prod sin(pi x_e), f = d pi^2 u; broken L2 error O(h^{k+1}), broken H1 O(h^k)
    def u(p):
        return np.prod(np.sin(np.pi * p), axis=1)

    def grad(p):
        g = np.zeros_like(p)
        for e in range(dim):
            g[:, e] = np.pi * np.cos(np.pi * p[:, e]) * np.prod(np.sin(np.pi * np.delete(p, e, axis=1)), axis=1)
        return g

    def f(p):
        return dim * np.pi ** 2 * u(p)

    errs = []
    for N in Ns:
        b = rhs_quadrature(dim, k, N, f)
        x = GlobalFD(dim, k, N).solve(b)
        errs.append(l2_error(dim, k, N, x, u, grad))
    l2 = np.array([e[0] for e in errs])
    h1 = np.array([e[1] for e in errs])
    r_l2 = np.log2(l2[:-1] / l2[1:])
    r_h1 = np.log2(h1[:-1] / h1[1:])
    assert r_l2[-1] > k + 1 - 0.25, (l2, r_l2)
    assert r_h1[-1] > k - 0.25, (h1, r_h1)
