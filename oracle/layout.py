"""Cell-wise lexicographic DoF numbering (paper Sec. 4.1, Fig. dof_layout right).

Test infrastructure only (see ``oracle/__init__.py``).

Cells of an N^d Cartesian mesh of the unit cube are numbered
c = c_0 + N c_1 + N^2 c_2 (x fastest); the n^d DoFs of a cell are contiguous
and lexicographic inside the cell, I = i_0 + n i_1 + n^2 i_2.  DoF (c, I) has
global index c * n^d + I.
"""
import numpy as np

from .basis import tensor_index


def cell_multi_index(dim, N):
    """(N^d, d) array of cell multi-indices (c_0 fastest)."""
    return tensor_index(dim, N)


def dof_index(dim, N, n, cells, local):
    """Global index of DoF ``local`` (flat, 0..n^d-1) of cell multi-index ``cells``."""
    cells = np.asarray(cells)
    c = np.zeros(cells.shape[:-1], dtype=np.int64)
    stride = 1
    for e in range(dim):
        c += cells[..., e] * stride
        stride *= N
    return c * n ** dim + np.asarray(local)


def cellwise_to_lex(dim, N, n):
    """perm such that x_lex = x_cell[perm]: the global lexicographic numbering
    (Fig. dof_layout left) X_e = c_e n + i_e, X_0 fastest, listed in
    lexicographic order, mapped to cell-wise indices."""
    m = N * n
    X = tensor_index(dim, m)                 # (m^d, d), X_0 fastest
    cells = X // n
    local = X % n
    loc = np.zeros(len(X), dtype=np.int64)
    stride = 1
    for e in range(dim):
        loc += local[:, e] * stride
        stride *= n
    return dof_index(dim, N, n, cells, loc)


def node_coordinates(dim, N, nodes1d):
    """(n_dofs, d) physical coordinates of the nodal DoFs on the unit cube,
    cell-wise lexicographic order."""
    n = len(nodes1d)
    h = 1.0 / N
    cells = cell_multi_index(dim, N)          # (N^d, d)
    local = tensor_index(dim, n)              # (n^d, d)
    xyz = (cells[:, None, :] + np.asarray(nodes1d)[local][None, :, :]) * h
    return xyz.reshape(-1, dim)
