"""SIPG discretisation of the Poisson problem (paper Sec. 2, Eqs. model,
jump_mean, jump_boundary, bilinear_form, weak_form, mat_form).

Test infrastructure only (see ``oracle/__init__.py``).

Generic d-dimensional quadrature assembly; it does NOT use the Kronecker
structure of Sec. 2.2 (that structure is what ``oracle.direct`` builds
independently, and the two are compared in the tests).

Conventions (readings of the paper where it is garbled or silent):
  * jump on an interior face: [[u]] = u^- n^- + u^+ n^+ (Eq. jump_mean prints
    "(u^+ + u^-) n^+", read as the standard SIPG jump); mean {g} = (g^- + g^+)/2;
  * boundary face: [[u]] = u n, {grad u} = grad u (Eq. jump_boundary);
  * penalty gamma_e = eta * k (k+1) (1/h^+ + 1/h^-) (Sec. 2.1) with eta = 1 the
    paper's value; on boundary faces h^- := h^+, i.e. gamma = 2 eta k (k+1) / h;
  * a scalar diffusion coefficient kappa multiplies the whole form;
  * exact Gauss quadrature (k+1 points per direction) for all bilinear forms.
"""
import numpy as np
import scipy.sparse as sp

from .basis import gauss, gauss_lobatto, lagrange_derivatives, lagrange_values, tensor_index
from .layout import cell_multi_index, dof_index


def penalty(k, N, eta=1.0):
    """gamma_e on a uniform mesh of cell size h = 1/N (Sec. 2.1)."""
    h = 1.0 / N
    return eta * k * (k + 1) * (1.0 / h + 1.0 / h)


def _tensor_points(dim, m):
    """m^dim tensor Gauss points on [0,1]^dim, weights; axis 0 fastest."""
    if dim == 0:
        return np.zeros((1, 0)), np.ones(1)
    x, w = gauss(m)
    idx = tensor_index(dim, m)
    pts = x[idx]
    wts = np.prod(w[idx], axis=1) if dim > 0 else np.ones(1)
    return pts, wts


def eval_basis(dim, k, h, y):
    """Values V[q, I] and physical gradients G[q, I, e] of the Q_k basis of a
    cell of size h at reference points y[q, :] in [0,1]^d (Appendix A)."""
    nodes, _ = gauss_lobatto(k)
    n = k + 1
    loc = tensor_index(dim, n)            # (n^d, d)
    y = np.atleast_2d(y)
    Q = y.shape[0]
    v1 = [lagrange_values(nodes, y[:, e]) for e in range(dim)]       # (Q, n)
    d1 = [lagrange_derivatives(nodes, y[:, e]) for e in range(dim)]  # (Q, n)
    V = np.ones((Q, n ** dim))
    for e in range(dim):
        V *= v1[e][:, loc[:, e]]
    G = np.ones((Q, n ** dim, dim))
    for g in range(dim):
        for e in range(dim):
            if e == g:
                G[:, :, g] *= d1[e][:, loc[:, e]] / h
            else:
                G[:, :, g] *= v1[e][:, loc[:, e]]
    return V, G


def cell_matrices(dim, k, N):
    """Cell stiffness int_K grad phi_J . grad phi_I and mass int_K phi_J phi_I
    (Sec. 2.1), tensor Gauss quadrature with k+1 points per direction."""
    h = 1.0 / N
    pts, wts = _tensor_points(dim, k + 1)
    V, G = eval_basis(dim, k, h, pts)
    jac = h ** dim
    K = jac * np.einsum("q,qie,qje->ij", wts, G, G)
    M = jac * np.einsum("q,qi,qj->ij", wts, V, V)
    return K, M


def _face_points(dim, k, e, s):
    """Quadrature on the face {y_e = s} of the reference cell: tangential
    tensor Gauss points (k+1 per tangential direction), returned as full
    d-dimensional reference coordinates."""
    tp, tw = _tensor_points(dim - 1, k + 1)
    pts = np.zeros((len(tw), dim))
    t = 0
    for f in range(dim):
        if f == e:
            pts[:, f] = s
        else:
            pts[:, f] = tp[:, t]
            t += 1
    return pts, tw


def face_matrices(dim, k, N, gamma, penalty_only=False, drop_last=False):
    """Face blocks of the SIPG form (Eq. bilinear_form) for every direction e.

    Returns a dict with, for each e:
      ('int', e): 2x2 nested list B[Y][X] (Y = test side, X = trial side,
                  0 = minus cell (face at its y_e = 1), 1 = plus cell (y_e = 0));
      ('bnd', e, s): block of a boundary face at y_e = s (s = 0: x_e = 0,
                  outward normal -e_e; s = 1: x_e = 1, normal +e_e).
    Entry [I, J] = int_F gamma [[phi_J]].[[phi_I]] - {grad phi_J}.[[phi_I]]
                   - [[phi_J]].{grad phi_I}  (or only the first term; with
    ``drop_last`` the first two, i.e. the last face term of Eq. bilinear_form
    left out).
    """
    h = 1.0 / N
    jac = h ** (dim - 1)
    out = {}
    for e in range(dim):
        unit = np.zeros(dim)
        unit[e] = 1.0
        # interior face: minus side sees it at y_e = 1, plus side at y_e = 0
        pm, w = _face_points(dim, k, e, 1.0)
        pp, _ = _face_points(dim, k, e, 0.0)
        Vs, Gs = zip(eval_basis(dim, k, h, pm), eval_basis(dim, k, h, pp))
        normals = [unit, -unit]           # outward normal of minus / plus cell
        # jump contribution of a basis function of side X: phi^X n^X (vector)
        jump = [Vs[X][:, :, None] * normals[X][None, None, :] for X in range(2)]
        avg = [0.5 * Gs[X] for X in range(2)]
        B = [[None, None], [None, None]]
        for Y in range(2):
            for X in range(2):
                pen = gamma * np.einsum("q,qje,qie->ij", w, jump[X], jump[Y])
                if penalty_only:
                    B[Y][X] = jac * pen
                else:
                    flux = np.einsum("q,qje,qie->ij", w, avg[X], jump[Y])
                    sym = 0.0 if drop_last else np.einsum("q,qje,qie->ij", w, jump[X], avg[Y])
                    B[Y][X] = jac * (pen - flux - sym)
        out[("int", e)] = B
        for s in (0, 1):
            pts, w = _face_points(dim, k, e, float(s))
            V, G = eval_basis(dim, k, h, pts)
            nvec = unit if s == 1 else -unit
            jmp = V[:, :, None] * nvec[None, None, :]
            pen = gamma * np.einsum("q,qje,qie->ij", w, jmp, jmp)
            if penalty_only:
                out[("bnd", e, s)] = jac * pen
            else:
                flux = np.einsum("q,qje,qie->ij", w, G, jmp)
                sym = 0.0 if drop_last else np.einsum("q,qje,qie->ij", w, jmp, G)
                out[("bnd", e, s)] = jac * (pen - flux - sym)
    return out


def element_blocks(dim, k, N, kappa=1.0, eta=1.0, part="full"):
    """All distinct element-level blocks of kappa * a_h on the uniform N^d mesh.

    part = "full": the whole form; "penalty": only sum_F int_F [[u]].[[v]]
    with gamma = 1 (the derivative of the form with respect to a uniform face
    penalty value), still multiplied by kappa; "no_last": the whole form
    without the last face term -[[u]].{grad v} (the face blocks the paper's
    Dirichlet kernel keeps on patch-boundary faces, Sec. 3.1)."""
    gamma = penalty(k, N, eta)
    if part in ("full", "no_last"):
        K, _ = cell_matrices(dim, k, N)
        F = face_matrices(dim, k, N, gamma, drop_last=(part == "no_last"))
    elif part == "penalty":
        n = k + 1
        K = np.zeros((n ** dim, n ** dim))
        F = face_matrices(dim, k, N, 1.0, penalty_only=True)
    else:
        raise ValueError(part)
    blocks = {"cell": kappa * K}
    for key, val in F.items():
        if key[0] == "int":
            blocks[key] = [[kappa * val[Y][X] for X in range(2)] for Y in range(2)]
        else:
            blocks[key] = kappa * val
    return blocks


def _scatter(rows_cells, cols_cells, block, dim, N, n, R, C, V):
    loc = np.arange(n ** dim)
    r = dof_index(dim, N, n, rows_cells[:, None, :], loc[None, :])  # (F, n^d)
    c = dof_index(dim, N, n, cols_cells[:, None, :], loc[None, :])
    F = len(rows_cells)
    R.append(np.broadcast_to(r[:, :, None], (F, n ** dim, n ** dim)).ravel())
    C.append(np.broadcast_to(c[:, None, :], (F, n ** dim, n ** dim)).ravel())
    V.append(np.broadcast_to(block[None], (F, n ** dim, n ** dim)).ravel())


def assemble(dim, k, N, kappa=1.0, eta=1.0, part="full"):
    """Global sparse matrix A of kappa * a_h (Eq. mat_form) in cell-wise
    lexicographic numbering: loop over cells and over interior and boundary
    faces of the N^d mesh, adding the blocks of ``element_blocks``."""
    n = k + 1
    blocks = element_blocks(dim, k, N, kappa, eta, part)
    cells = cell_multi_index(dim, N)
    R, C, V = [], [], []
    _scatter(cells, cells, blocks["cell"], dim, N, n, R, C, V)
    for e in range(dim):
        minus = cells[cells[:, e] < N - 1]
        plus = minus.copy()
        plus[:, e] += 1
        side = [minus, plus]
        B = blocks[("int", e)]
        for Y in range(2):
            for X in range(2):
                _scatter(side[Y], side[X], B[Y][X], dim, N, n, R, C, V)
        for s, sel in ((0, cells[:, e] == 0), (1, cells[:, e] == N - 1)):
            cs = cells[sel]
            _scatter(cs, cs, blocks[("bnd", e, s)], dim, N, n, R, C, V)
    ndof = N ** dim * n ** dim
    A = sp.coo_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(C))),
                      shape=(ndof, ndof)).tocsr()
    A.sum_duplicates()
    A.eliminate_zeros()
    return A


def block_apply(dim, k, N, blocks, x, cells_sel=None):
    """y = A x evaluated cell by cell from the element blocks, for the cells
    listed in ``cells_sel`` (flat cell numbers; default all).  Returns the
    (len(cells_sel), n^d) rows of y.  Same numbers as ``assemble`` without
    building the global matrix, for meshes too large to assemble."""
    n = k + 1
    nloc = n ** dim
    allc = cell_multi_index(dim, N)
    if cells_sel is None:
        cells_sel = np.arange(N ** dim)
    cells_sel = np.asarray(cells_sel, dtype=np.int64)
    cm = allc[cells_sel]
    X = np.asarray(x, dtype=np.float64).reshape(N ** dim, nloc)
    y = X[cells_sel] @ blocks["cell"].T
    strides = N ** np.arange(dim)
    for e in range(dim):
        B = blocks[("int", e)]
        lo = cm[:, e] > 0
        hi = cm[:, e] < N - 1
        # face on the low side: this cell is the plus side (index 1)
        nb = cells_sel - strides[e]
        y[lo] += X[cells_sel[lo]] @ B[1][1].T + X[nb[lo]] @ B[1][0].T
        y[~lo] += X[cells_sel[~lo]] @ blocks[("bnd", e, 0)].T
        # face on the high side: this cell is the minus side (index 0)
        nb = cells_sel + strides[e]
        y[hi] += X[cells_sel[hi]] @ B[0][0].T + X[nb[hi]] @ B[0][1].T
        y[~hi] += X[cells_sel[~hi]] @ blocks[("bnd", e, 1)].T
    return y


def principal_block(dim, k, N, blocks, cells_sel, outer=None):
    """Dense A[D, D] for D = all DoFs of the listed cells (flat cell numbers,
    in the given order, n^d DoFs each), from the element blocks: a cell's
    diagonal block is its cell block plus the self parts of its faces; two
    listed cells sharing a face couple through that face's off-diagonal block.
    For the vertex-patch cells this is the patch matrix of Sec. 3.1 before
    restriction to V_j, on meshes too large to assemble.

    ``outer``: element blocks used instead of ``blocks`` for the self part of
    a face whose other cell is NOT listed (an interior mesh face on the
    boundary of the selection); faces on the domain boundary keep ``blocks``.
    With ``element_blocks(..., part="no_last")`` this gives the patch operator
    of the paper's Dirichlet kernel (Sec. 3.1)."""
    if outer is None:
        outer = blocks
    n = k + 1
    nl = n ** dim
    allc = cell_multi_index(dim, N)
    cells_sel = [int(c) for c in cells_sel]
    pos = {c: i for i, c in enumerate(cells_sel)}
    out = np.zeros((len(cells_sel) * nl, len(cells_sel) * nl))
    strides = N ** np.arange(dim)
    for i, c in enumerate(cells_sel):
        cm = allc[c]
        D = blocks["cell"].copy()
        for e in range(dim):
            B = blocks[("int", e)]
            if cm[e] > 0:
                j = pos.get(c - int(strides[e]))
                if j is not None:
                    D += B[1][1]
                    out[i * nl:(i + 1) * nl, j * nl:(j + 1) * nl] += B[1][0]
                else:
                    D += outer[("int", e)][1][1]
            else:
                D += blocks[("bnd", e, 0)]
            if cm[e] < N - 1:
                j = pos.get(c + int(strides[e]))
                if j is not None:
                    D += B[0][0]
                    out[i * nl:(i + 1) * nl, j * nl:(j + 1) * nl] += B[0][1]
                else:
                    D += outer[("int", e)][0][0]
            else:
                D += blocks[("bnd", e, 1)]
        out[i * nl:(i + 1) * nl, i * nl:(i + 1) * nl] += D
    return out


def mass_matrix_cell(dim, k, N):
    """Exact cell mass matrix (k+1 Gauss points per direction)."""
    return cell_matrices(dim, k, N)[1]


def rhs_from_nodal(dim, k, N, f_nodal):
    """b = M_h f for a source given by its nodal values in V_h (the reading of
    Eq. weak_form used for seeded and manufactured sources): the block
    diagonal exact mass matrix applied cell by cell."""
    n = k + 1
    M = mass_matrix_cell(dim, k, N)
    F = np.asarray(f_nodal, dtype=np.float64).reshape(N ** dim, n ** dim)
    return (F @ M.T).ravel()


def mass_apply(dim, k, N, v):
    """M_h v (block diagonal exact mass)."""
    return rhs_from_nodal(dim, k, N, v)


def rhs_quadrature(dim, k, N, f):
    """b_I = sum_K int_K f phi_I with k+2 Gauss points per direction
    (Eq. weak_form evaluated without interpolating f)."""
    h = 1.0 / N
    pts, wts = _tensor_points(dim, k + 2)
    V, _ = eval_basis(dim, k, h, pts)
    cells = cell_multi_index(dim, N)
    xq = (cells[:, None, :] + pts[None, :, :]) * h          # (cells, Q, d)
    fq = f(xq.reshape(-1, dim)).reshape(len(cells), len(wts))
    b = (h ** dim) * (fq * wts[None, :]) @ V               # (cells, n^d)
    return b.ravel()


def l2_error(dim, k, N, x, u_exact, grad_exact=None):
    """Broken L2 (and optionally broken H1-seminorm) error of the discrete
    function with nodal values x against u_exact, (k+3)-point Gauss."""
    h = 1.0 / N
    n = k + 1
    pts, wts = _tensor_points(dim, k + 3)
    V, G = eval_basis(dim, k, h, pts)
    cells = cell_multi_index(dim, N)
    X = np.asarray(x).reshape(N ** dim, n ** dim)
    xq = ((cells[:, None, :] + pts[None, :, :]) * h).reshape(-1, dim)
    uh = (X @ V.T).ravel()
    err = uh - u_exact(xq)
    l2 = np.sqrt(h ** dim * np.sum(err.reshape(len(cells), -1) ** 2 * wts[None, :]))
    if grad_exact is None:
        return l2
    gh = np.einsum("cj,qje->cqe", X, G).reshape(-1, dim)
    gerr = gh - grad_exact(xq)
    h1 = np.sqrt(h ** dim * np.sum(np.sum(gerr ** 2, axis=1).reshape(len(cells), -1) * wts[None, :]))
    return l2, h1
