"""1D ingredients of the Q_k tensor basis (paper Appendix A).

Test infrastructure only (see ``oracle/__init__.py``).

The 1D shape functions are the Lagrange polynomials on the k+1 Gauss-Lobatto
points of the reference interval [0, 1] (Appendix A): phi_nu(xi_mu) =
delta_{mu nu}.  The d-dimensional basis is their tensor product, x index
fastest.
"""
import numpy as np


def legendre(k, x):
    """Return (P_k(x), P_{k-1}(x)) by the three-term recurrence
    m P_m = (2m-1) x P_{m-1} - (m-1) P_{m-2}.  Requires k >= 1."""
    x = np.asarray(x, dtype=np.float64)
    p_prev = np.ones_like(x)
    p = x.copy()
    for m in range(2, k + 1):
        p_prev, p = p, ((2 * m - 1) * x * p - (m - 1) * p_prev) / m
    return p, p_prev


def gauss_lobatto(k):
    """k+1 Gauss-Lobatto points and weights on [0, 1] (Appendix A).

    The points are -1, 1 and the roots of P_k' on [-1, 1], mapped to [0, 1].
    Newton's method is applied to q(x) = (1 - x^2) P_k'(x) = k (P_{k-1} - x P_k),
    whose derivative is -k (k+1) P_k by Legendre's equation, giving the update
    x <- x - (x P_k - P_{k-1}) / ((k+1) P_k); the end points are fixed points.
    Start: Chebyshev-Gauss-Lobatto points.  Weights on [-1, 1] are
    2 / (k (k+1) P_k(x_i)^2); halved for [0, 1].
    """
    if k < 1:
        raise ValueError("Gauss-Lobatto rule needs k >= 1")
    x = -np.cos(np.pi * np.arange(k + 1) / k)
    for _ in range(100):
        p, pm1 = legendre(k, x)
        dx = (x * p - pm1) / ((k + 1) * p)
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    p, _ = legendre(k, x)
    w = 2.0 / (k * (k + 1) * p * p)
    return 0.5 * (x + 1.0), 0.5 * w


def gauss(m):
    """m-point Gauss-Legendre rule on [0, 1] (library routine, mapped)."""
    x, w = np.polynomial.legendre.leggauss(m)
    return 0.5 * (x + 1.0), 0.5 * w


def lagrange_values(nodes, x):
    """V[q, j] = phi_j(x_q) for the Lagrange basis on ``nodes``.

    phi_j(x) = prod_{m != j} (x - xi_m) / (xi_j - xi_m)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    V = np.ones((len(x), n))
    for j in range(n):
        for m in range(n):
            if m != j:
                V[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
    return V


def lagrange_derivatives(nodes, x):
    """D[q, j] = phi_j'(x_q): product rule over the factors of phi_j,
    phi_j'(x) = sum_{l != j} 1/(xi_j - xi_l) prod_{m != j, l} (x - xi_m)/(xi_j - xi_m)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    D = np.zeros((len(x), n))
    for j in range(n):
        for l in range(n):
            if l == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[l]))
            for m in range(n):
                if m != j and m != l:
                    term *= (x - nodes[m]) / (nodes[j] - nodes[m])
            D[:, j] += term
    return D


def tensor_index(dim, n):
    """Multi-indices (i_0, ..., i_{d-1}) of the n^d tensor basis, in
    lexicographic order with i_0 fastest (cell-wise lexicographic numbering
    inside a cell, Sec. 4.1).  Returns an (n^d, d) integer array."""
    idx = np.indices((n,) * dim).reshape(dim, -1).T  # last axis fastest
    return idx[:, ::-1].copy()                        # make axis 0 fastest
