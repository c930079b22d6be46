"""Kronecker form of the SIPG matrix and the global fast-diagonalisation
direct solver (paper Sec. 2.2 and Sec. 3.2, Eqs. inverse2d, inverse3d,
fast_inverse).

Test infrastructure only (see ``oracle/__init__.py``).

On a uniform Cartesian mesh with constant coefficient the whole d-dimensional
SIPG matrix, faces included, in global lexicographic numbering (Fig.
dof_layout left) is a Kronecker sum of the 1D DG matrices (Sec. 2.2 states it
per cell; the face terms factor the same way because a face integral is a 1D
point term times tangential 1D masses):

    A_lex = sum_e  M (x) ... (x) L (in slot e) (x) ... (x) M,

with L the 1D SIPG matrix (size N n) and M the 1D block-diagonal mass, slot 0
the fastest index.  Its inverse is (S (x) ... (x) S) D^{-1} (S^T (x) ... (x) S^T)
with L S = M S Lambda, S^T M S = I and D = sum of the Lambdas (Eq.
fast_inverse).  This gives an exact solver independent of multigrid.
"""
import numpy as np
import scipy.linalg as sla

from .assembly import assemble
from .layout import cellwise_to_lex


def one_d_matrices(k, N, kappa=1.0, eta=1.0):
    """1D SIPG matrix L and mass M on N cells of [0,1] (dense), built by the
    generic assembly in dimension 1 (Sec. 2.1 with d = 1)."""
    L = assemble(1, k, N, kappa, eta).toarray()
    from .assembly import mass_matrix_cell
    Mc = mass_matrix_cell(1, k, N)
    M = np.kron(np.eye(N), Mc)
    return L, M


def kron_sum(dim, L, M):
    """A_lex = sum_e (x)_{f = d-1..0} (L if f == e else M) (slot 0 fastest)."""
    total = None
    for e in range(dim):
        term = np.ones((1, 1))
        for f in reversed(range(dim)):
            term = np.kron(term, L if f == e else M)
        total = term if total is None else total + term
    return total


class GlobalFD:
    """Exact solve of A x = b through the 1D generalised eigenproblem
    L S = M S Lambda (scipy.linalg.eigh, M-orthonormal S)."""

    def __init__(self, dim, k, N, kappa=1.0, eta=1.0):
        self.dim, self.k, self.N = dim, k, N
        self.n = k + 1
        L, M = one_d_matrices(k, N, kappa, eta)
        lam, S = sla.eigh(L, M)
        self.lam, self.S = lam, S
        self.perm = cellwise_to_lex(dim, N, self.n)
        m = N * self.n
        grids = np.meshgrid(*([lam] * dim), indexing="ij")   # axis order (slot d-1, ..., slot 0)
        self.D = sum(grids)
        self.m = m

    def _modes(self, X, Mat):
        """Apply Mat along every axis of the lexicographic tensor X."""
        for ax in range(self.dim):
            X = np.moveaxis(np.tensordot(Mat, X, axes=([1], [ax])), 0, ax)
        return X

    def solve(self, b):
        m, d = self.m, self.dim
        blex = np.asarray(b, dtype=np.float64)[self.perm].reshape((m,) * d)
        y = self._modes(blex, self.S.T)
        y = y / self.D
        x = self._modes(y, self.S)
        out = np.empty(m ** d)
        out[self.perm] = x.ravel()
        return out
