"""Pins of the oracle's 1D basis (Appendix A) against closed forms and an
independent library routine."""
import numpy as np
import pytest

from oracle.basis import gauss, gauss_lobatto, lagrange_derivatives, lagrange_values


CLOSED_FORM_NODES = {
    1: [0.0, 1.0],
    2: [0.0, 0.5, 1.0],
    3: [0.0, 0.5 * (1 - 1 / np.sqrt(5)), 0.5 * (1 + 1 / np.sqrt(5)), 1.0],
    4: [0.0, 0.5 * (1 - np.sqrt(3 / 7)), 0.5, 0.5 * (1 + np.sqrt(3 / 7)), 1.0],
}
# weights on [-1, 1] (textbook values), halved for [0, 1]
CLOSED_FORM_WEIGHTS = {
    2: [1 / 3, 4 / 3, 1 / 3],
    3: [1 / 6, 5 / 6, 5 / 6, 1 / 6],
    4: [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10],
}


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_gll_closed_form(k):
    x, w = gauss_lobatto(k)
    assert np.allclose(x, CLOSED_FORM_NODES[k], atol=1e-15, rtol=0)
    if k in CLOSED_FORM_WEIGHTS:
        assert np.allclose(w, 0.5 * np.array(CLOSED_FORM_WEIGHTS[k]), atol=1e-15, rtol=0)


@pytest.mark.parametrize("k", [2, 3, 4, 5, 6, 7])
def test_gll_interior_are_roots_of_legendre_derivative(k):
    # independent: numpy's Legendre class, roots of P_k'
    roots = np.sort(np.polynomial.legendre.Legendre.basis(k).deriv().roots().real)
    x, _ = gauss_lobatto(k)
    assert np.allclose(x[1:-1], 0.5 * (roots + 1), atol=1e-13, rtol=0)
    assert x[0] == 0.0 and x[-1] == 1.0


@pytest.mark.parametrize("k", [1, 2, 3, 5, 7])
def test_gll_quadrature_exact_to_degree_2k_minus_1(k):
    x, w = gauss_lobatto(k)
    for m in range(2 * k):
        assert abs(w @ x ** m - 1.0 / (m + 1)) < 1e-14
    # and not exact for degree 2k (Lobatto rules lose one degree)
    assert abs(w @ x ** (2 * k) - 1.0 / (2 * k + 1)) > 1e-11


@pytest.mark.parametrize("m", [1, 3, 8, 9])
def test_gauss_exact_to_degree_2m_minus_1(m):
    x, w = gauss(m)
    for p in range(2 * m):
        assert abs(w @ x ** p - 1.0 / (p + 1)) < 1e-14


@pytest.mark.parametrize("k", [1, 2, 3, 4, 7])
def test_lagrange_interpolation_properties(k):
    nodes, _ = gauss_lobatto(k)
    V = lagrange_values(nodes, nodes)
    assert np.allclose(V, np.eye(k + 1), atol=1e-14)
    t = np.linspace(-0.3, 1.2, 41)
    Vt = lagrange_values(nodes, t)
    Dt = lagrange_derivatives(nodes, t)
    assert np.allclose(Vt.sum(axis=1), 1.0, atol=1e-12)
    assert np.allclose(Dt.sum(axis=1), 0.0, atol=1e-10)
    # polynomials of degree <= k are reproduced, with their derivatives
    for p in range(k + 1):
        assert np.allclose(Vt @ nodes ** p, t ** p, atol=1e-12)
        dp = p * t ** (p - 1) if p > 0 else np.zeros_like(t)
        assert np.allclose(Dt @ nodes ** p, dp, atol=1e-10)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7])
def test_exact_gll_mass_is_diagonal_plus_rank_one(k):
    # the n-point GLL rule is exact up to degree 2n-3, phi_i phi_j has degree
    # 2n-2, so M_ij - w_i delta_ij = E(x^(2k)) lead(phi_i) lead(phi_j): the
    # exact mass minus the GLL weights is a rank-one matrix built from the
    # leading coefficients 1 / prod_{m != i} (xi_i - xi_m)
    from oracle.assembly import mass_matrix_cell
    xi, w = gauss_lobatto(k)
    M = mass_matrix_cell(1, k, 1)
    lead = np.array([1.0 / np.prod([xi[i] - xi[m] for m in range(k + 1) if m != i]) for i in range(k + 1)])
    R = M - np.diag(w)
    e = R[0, k] / (lead[0] * lead[k])
    assert np.abs(R - e * np.outer(lead, lead)).max() < 1e-13 * np.abs(M).max()
    assert np.linalg.matrix_rank(R, tol=1e-10 * np.abs(R).max()) == 1
