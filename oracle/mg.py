"""Multigrid preconditioner with the colourised vertex-patch smoother and the
outer flexible CG (paper Sec. 3, Sec. 3.1 Algorithm 1, Eqs. residual and
local-solver; Sec. 3.3 for the iteration count nu).

Test infrastructure only (see ``oracle/__init__.py``).

Readings of the paper (where it is silent or ambiguous):
  * level l has N_l = N_L / 2^(L-l) cells per direction; the coarsest level
    is solved exactly (P_0^{-1} = A_0^{-1}, Sec. 3);
  * coarse operators are re-discretised SIPG matrices with their own h;
  * prolongation is the canonical embedding (Sec. 3): fine nodal values are
    the coarse polynomial evaluated at the fine nodes; restriction of
    residuals is its transpose P^T (the L2-projection of Sec. 3 seen on dual
    vectors);
  * one patch per interior vertex, the 2^d cells sharing it (Sec. 3.1);
  * Dirichlet kernel space V_j: all nodes of the patch cells except the
    nodes on the patch boundary (Sec. 3.1); a patch-boundary end that lies on
    the domain boundary is kept in V_j (the paper is silent);
  * "consistent" local residual r_j = R_j (b - A x) (default), or the paper's
    Dirichlet-kernel residual r_j = R_j b - Abar_j Rbar_j x ("paper"): Abar_j
    is the form on the patch cells alone (cell terms, all terms of the faces
    between patch cells and on the domain boundary) in which the last face
    term -[[u]].{grad v} of the patch-boundary faces inside the domain is
    left out.  Sec. 3.1 states that this term does not vanish for v in V_j
    and that ignoring it makes the residual inconsistent; keeping its
    patch-side half instead gives iteration counts that grow with the level,
    unlike Table 2;
  * the paper's clamped kernel ("clamped", Sec. 3.1, Table 2 right): V_j is
    the functions on the patch cells whose value and normal derivative vanish
    on the patch boundary inside the domain (no condition at a patch end on
    the domain boundary, as for the Dirichlet kernel), (2k-2)^d functions for
    an interior patch.  The paper spans it by a Hermite-type basis; here it is
    the same space written in the Lagrange basis (an orthonormal basis of the
    null space of the end conditions per direction, tensorised), so the
    correction x += B (B^T A_D B)^{-1} B^T R_D (b - A x) is the paper's, while
    the Euclidean residual norm of the outer solver (and hence nu) is that of
    the Lagrange basis.  All patch-boundary face terms vanish for these test
    functions, so the residual needs only the patch cells and is exact;
  * the paper's full kernel ("full", Sec. 3.1, Table 1): V_j is every DoF of
    the 2^d patch cells and A_j the principal block of A on them; the residual
    is updated globally once per colour (r = b - A x), and every patch of the
    colour adds A_j^{-1} R_j r.  Same-colour patches share faces but no DoFs,
    so inside a colour the corrections are additive;
  * colours: c = sum_e (v_e mod 2) 2^e for vertex index v; pre-smoothing visits
    colours 0..2^d-1, post-smoothing visits them in reverse;
  * outer solver: flexible CG with beta = <z_{i+1}, r_{i+1} - r_i> / <z_i, r_i>,
    stopped at ||r||_2 / ||b||_2 <= rtol (Euclidean norm, Sec. 3.3), or the
    paper's GMRES (Sec. 3.3, Tables 1 and 2), preconditioned from the right so
    that its residual is the Euclidean residual of Ax = b.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .assembly import assemble, element_blocks, principal_block
from .basis import gauss_lobatto, lagrange_derivatives, lagrange_values, tensor_index
from .layout import cell_multi_index, dof_index


# ---------------------------------------------------------------- transfer
def prolongation(dim, k, Nc):
    """Sparse P from the coarse mesh (Nc^d cells) to the fine mesh (2Nc)^d:
    P[(f, I), (C, J)] = Phi_J(y_I) where fine cell f = 2C + o, o in {0,1}^d,
    and y_I = (o + xi_I) / 2 are the fine node coordinates in the coarse
    reference cell (canonical embedding, Sec. 3)."""
    n = k + 1
    nodes, _ = gauss_lobatto(k)
    loc = tensor_index(dim, n)                 # (n^d, d)
    Nf = 2 * Nc
    coarse = cell_multi_index(dim, Nc)
    offsets = tensor_index(dim, 2)
    R, C, V = [], [], []
    for o in offsets:
        y = (o[None, :] + nodes[loc]) / 2.0   # (n^d, d) fine nodes in coarse coords
        E = np.ones((n ** dim, n ** dim))      # E[I, J] = Phi_J(y_I)
        for e in range(dim):
            E *= lagrange_values(nodes, y[:, e])[:, loc[:, e]]
        fine = 2 * coarse + o[None, :]
        r = dof_index(dim, Nf, n, fine[:, None, :], np.arange(n ** dim)[None, :])
        c = dof_index(dim, Nc, n, coarse[:, None, :], np.arange(n ** dim)[None, :])
        F = len(coarse)
        R.append(np.broadcast_to(r[:, :, None], (F, n ** dim, n ** dim)).ravel())
        C.append(np.broadcast_to(c[:, None, :], (F, n ** dim, n ** dim)).ravel())
        V.append(np.broadcast_to(E[None], (F, n ** dim, n ** dim)).ravel())
    P = sp.coo_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(C))),
                      shape=(Nf ** dim * n ** dim, Nc ** dim * n ** dim)).tocsr()
    P.eliminate_zeros()
    return P


# ---------------------------------------------------------------- patches
def clamped_basis_1d(k, lo_on_boundary, hi_on_boundary):
    """(2n, m) orthonormal basis of the 1D clamped patch space in the Lagrange
    coefficients of the two patch cells: the null space of the conditions
    v = 0 and v' = 0 at each patch end that is not on the domain boundary
    (Sec. 3.1, clamped kernel).  m = 2k - 2 for an interior patch."""
    n = k + 1
    nodes, _ = gauss_lobatto(k)
    val0 = lagrange_values(nodes, np.array([0.0]))[0]
    val1 = lagrange_values(nodes, np.array([1.0]))[0]
    der0 = lagrange_derivatives(nodes, np.array([0.0]))[0]
    der1 = lagrange_derivatives(nodes, np.array([1.0]))[0]
    rows = []
    if not lo_on_boundary:                      # low end of cell 0
        for f in (val0, der0):
            r = np.zeros(2 * n)
            r[:n] = f
            rows.append(r)
    if not hi_on_boundary:                      # high end of cell 1
        for f in (val1, der1):
            r = np.zeros(2 * n)
            r[n:] = f
            rows.append(r)
    if not rows:
        return np.eye(2 * n)
    return sla.null_space(np.array(rows))


def vertex_patches(dim, k, N, variant="consistent"):
    """All vertex patches of the N^d mesh (one per interior vertex).

    Returns a list of dicts with keys
      vertex  : vertex multi-index v (each v_e in 1..N-1)
      colour  : sum_e (v_e mod 2) 2^e
      V       : sorted global DoF indices of the Dirichlet-kernel space V_j
      dofs    : all DoF indices of the 2^d patch cells (domain of dependence
                of the paper's Dirichlet kernel)
      cells   : the flat numbers of the 2^d patch cells, ascending (their DoFs
                in this order are ``dofs``)
      type    : per direction (v_e == 1, v_e == N-1)
    """
    n = k + 1
    nloc = n ** dim
    loc = tensor_index(dim, n)
    offsets = tensor_index(dim, 2)
    patches = []
    for v in tensor_index(dim, N - 1) + 1:
        keepV, alld, cells = [], [], []
        for o in offsets:
            cell = v - 1 + o
            cells.append(int(sum(int(cell[e]) * N ** e for e in range(dim))))
            g = dof_index(dim, N, n, cell[None, :], np.arange(nloc))
            a = o[None, :] * n + loc                  # 1D patch coordinates 0..2n-1
            inside = np.ones(nloc, dtype=bool)
            for e in range(dim):
                left_ok = (a[:, e] != 0) | (v[e] == 1)
                right_ok = (a[:, e] != 2 * n - 1) | (v[e] == N - 1)
                inside &= left_ok & right_ok
            keepV.append(g[inside])
            alld.append(g)
        patches.append(dict(
            vertex=tuple(int(t) for t in v),
            colour=int(sum((int(v[e]) % 2) << e for e in range(dim))),
            V=np.sort(np.concatenate(keepV)),
            dofs=np.sort(np.concatenate(alld)),
            cells=sorted(cells),
            type=tuple((bool(v[e] == 1), bool(v[e] == N - 1)) for e in range(dim)),
        ))
    return patches


class Level:
    """One level of the hierarchy: matrix, patches and their local solvers."""

    def __init__(self, dim, k, N, kappa=1.0, eta=1.0, variant="consistent"):
        self.dim, self.k, self.N = dim, k, N
        self.variant = variant
        self.A = assemble(dim, k, N, kappa, eta)
        self.ndof = self.A.shape[0]
        self.patches = vertex_patches(dim, k, N)
        if variant == "paper":
            full = element_blocks(dim, k, N, kappa, eta)
            no_last = element_blocks(dim, k, N, kappa, eta, part="no_last")
        factors = {}
        for p in self.patches:
            p["B"] = None
            if variant in ("full", "clamped"):
                p["V"] = p["dofs"]                   # every DoF of the patch cells
            V = p["V"]
            Aj = self.A[V][:, V].toarray()           # A_j = R_j A R_j^T
            if variant == "clamped":
                if k < 2:
                    raise ValueError("the clamped kernel needs k >= 2")
                p["B"] = self._clamped_basis(p)
                Aj = p["B"].T @ Aj @ p["B"]          # A on the clamped space
            if variant in ("full", "clamped"):
                # patches of one type have equal A_j on the uniform mesh: the
                # (large) factor is kept once per type, after checking that
                p["rows"], p["cols"] = self.A[V], None
                if p["type"] in factors:
                    A0, f0 = factors[p["type"]]
                    if np.abs(Aj - A0).max() > 1e-13 * np.abs(A0).max():
                        raise AssertionError("patches of one type differ")
                    p["chol"] = f0
                else:
                    p["chol"] = sla.cho_factor(Aj, lower=True)
                    factors[p["type"]] = (Aj, p["chol"])
                continue
            p["chol"] = sla.cho_factor(Aj, lower=True)
            if variant in ("consistent", "full"):
                p["rows"] = self.A[V]                # all columns: R_j A
                p["cols"] = None
            elif variant == "paper":
                # Abar_j over the patch cells, rows V_j: the last face term
                # dropped on the patch-boundary faces inside the domain
                Abar = principal_block(dim, k, N, full, p["cells"], outer=no_last)
                p["rows"] = Abar[np.searchsorted(p["dofs"], V)]
                p["cols"] = p["dofs"]
            else:
                raise ValueError(variant)

    def _clamped_basis(self, p):
        """Tensor product of the 1D clamped bases, rows in the order of
        p["dofs"] (cell-wise lexicographic)."""
        dim, k, N = self.dim, self.k, self.N
        n = k + 1
        v = p["vertex"]
        B1 = [clamped_basis_1d(k, v[e] == 1, v[e] == N - 1) for e in range(dim)]
        B = np.ones((1, 1))
        for e in range(dim - 1, -1, -1):            # patch-lexicographic, direction 0 fastest
            B = np.kron(B, B1[e])
        out = np.zeros((len(p["dofs"]), B.shape[1]))
        for row, t in enumerate(np.ndindex(*(2 * n,) * dim)):
            a = t[::-1]                              # (a_0, a_1, ...), a_0 fastest
            cell = sum((v[e] - 1 + a[e] // n) * N ** e for e in range(dim))
            node = sum((a[e] % n) * n ** e for e in range(dim))
            out[np.searchsorted(p["dofs"], cell * n ** dim + node)] = B[row]
        return out

    def colour_order(self, reverse=False):
        order = list(range(2 ** self.dim))
        return order[::-1] if reverse else order


def local_residual(patch, b, x):
    """r_j of Algorithm 1 (consistent: R_j (b - A x); paper: R_j b - Abar_j Rbar_j x)."""
    V = patch["V"]
    if patch["cols"] is None:
        return b[V] - patch["rows"] @ x
    return b[V] - patch["rows"] @ x[patch["cols"]]


def smooth(level, x, b, reverse=False, patch_order=None, colours=None):
    """One step of the colourised multiplicative vertex-patch smoother
    S_l(x, b) (Algorithm 1): colours in sequence; inside a colour, patches
    one after another (the paper's parallel loop; the tests check that the
    order inside a colour does not change the result), each doing
    r_j <- local residual; x <- x + R_j^T A_j^{-1} r_j (for the full kernel
    the residual of the whole colour is computed once before its patches;
    for the clamped kernel A_j and the correction live in the span of the
    patch's clamped basis B).
    ``colours`` restricts the sweep to the listed colours (in that order)."""
    x = np.array(x, dtype=np.float64, copy=True)
    order = level.colour_order(reverse) if colours is None else list(colours)
    for c in order:
        members = [p for p in level.patches if p["colour"] == c]
        if patch_order is not None:
            members = [members[i] for i in patch_order(c, len(members))]
        if level.variant == "full":
            # full kernel: one global residual per colour, additive inside it
            r = b - level.A @ x
            for p in members:
                x[p["V"]] += sla.cho_solve(p["chol"], r[p["V"]])
            continue
        for p in members:
            r = local_residual(p, b, x)
            if p["B"] is None:
                x[p["V"]] += sla.cho_solve(p["chol"], r)
            else:                                    # clamped: correction in span(B)
                x[p["V"]] += p["B"] @ sla.cho_solve(p["chol"], p["B"].T @ r)
    return x


class Hierarchy:
    """Mesh hierarchy T_0 < ... < T_L with N_l = N_L / 2^(L-l) (Sec. 3)."""

    def __init__(self, dim, k, N, n_levels, kappa=1.0, eta=1.0, variant="consistent"):
        if N % (1 << (n_levels - 1)) != 0 or N >> (n_levels - 1) < 2:
            raise ValueError("coarsest level needs >= 2 cells per direction")
        self.dim, self.k, self.N, self.L = dim, k, N, n_levels - 1
        self.levels = []
        self.P = [None]
        for l in range(n_levels):
            Nl = N >> (self.L - l)
            self.levels.append(Level(dim, k, Nl, kappa, eta, variant))
            if l > 0:
                self.P.append(prolongation(dim, k, Nl // 2))
        A0 = self.levels[0].A.toarray()
        self.coarse = sla.cho_factor(A0, lower=True)

    def vcycle(self, b, l=None):
        """Action of the multigrid preconditioner P_l^{-1} on b (Sec. 3):
        pre-smoothing from x = 0, coarse-grid correction
        x += I^up P_{l-1}^{-1} I^down (b - A_l x), post-smoothing (reversed
        colours); P_0^{-1} = A_0^{-1}."""
        if l is None:
            l = self.L
        if l == 0:
            return sla.cho_solve(self.coarse, b)
        lev = self.levels[l]
        x = np.zeros(lev.ndof)
        x = smooth(lev, x, b, reverse=False)
        r = b - lev.A @ x
        rc = self.P[l].T @ r
        ec = self.vcycle(rc, l - 1)
        x = x + self.P[l] @ ec
        x = smooth(lev, x, b, reverse=True)
        return x

    @property
    def A(self):
        return self.levels[-1].A


def fcg(A_apply, precond, b, rtol=1e-10, maxit=200, x0=None):
    """Flexible preconditioned CG (Polak-Ribiere form):
      r_0 = b - A x_0, z_0 = B r_0, p_0 = z_0;
      alpha_i = <r_i, z_i> / <p_i, A p_i>; x += alpha p; r -= alpha A p;
      z_{i+1} = B r_{i+1}; beta_i = <z_{i+1}, r_{i+1} - r_i> / <z_i, r_i>;
      p_{i+1} = z_{i+1} + beta_i p_i.
    Stops when ||r||_2 <= rtol ||b||_2.  Returns (x, history of ||r||_2)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - A_apply(x)
    bnorm = np.linalg.norm(b)
    hist = [np.linalg.norm(r)]
    if bnorm == 0.0 or hist[0] <= rtol * bnorm:
        return x, hist
    z = precond(r)
    p = z.copy()
    rz = r @ z
    for _ in range(maxit):
        q = A_apply(p)
        alpha = rz / (p @ q)
        x = x + alpha * p
        r_new = r - alpha * q
        hist.append(np.linalg.norm(r_new))
        if hist[-1] <= rtol * bnorm:
            break
        z_new = precond(r_new)
        beta = (z_new @ (r_new - r)) / rz
        p = z_new + beta * p
        r, z = r_new, z_new
        rz = r @ z
    return x, hist


def gmres(A_apply, precond, b, rtol=1e-8, maxit=200, restart=30, x0=None, side="right"):
    """GMRES preconditioned from the right (side="right") or from the left
    (side="left": GMRES on B A x = B b with the preconditioned residual
    B (b - A x) as its residual, norm and stopping test ||B r|| <= rtol
    ||B b||, the reading of Table 2's clamped column).

    Right preconditioning in its flexible form (the
    preconditioned directions z_j = B v_j are kept, so B may vary between
    steps; for a fixed B this is right-preconditioned GMRES).  Arnoldi with
    modified Gram-Schmidt builds an orthonormal basis v_1..v_{j+1} with
    A z_j = sum_i h_ij v_i; plane rotations reduce the Hessenberg matrix to
    triangular form, so that |g_{j+1}| is the Euclidean norm of b - A x_j for
    the x_j = x_0 + Z_j y_j minimising it.  A cycle ends after ``restart``
    steps or when that norm reaches rtol ||b||_2; then x is updated and the
    true residual b - A x recomputed (it replaces the last history entry):
    the solve stops when it is <= rtol ||b||_2, else GMRES restarts from x.
    Returns (x, history of ||r||_2), the history starting with ||r_0||."""
    if side == "left":
        return gmres(lambda v: precond(A_apply(v)), lambda r: r, precond(np.asarray(b, dtype=np.float64)),
                     rtol, maxit, restart, x0, "right")
    if side != "right":
        raise ValueError(side)
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    r = b - A_apply(x)
    hist = [np.linalg.norm(r)]
    if bnorm == 0.0 or hist[0] <= rtol * bnorm:
        return x, hist
    steps = 0
    while steps < maxit:
        beta = np.linalg.norm(r)
        m = min(restart, maxit - steps)
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m))
        g = np.zeros(m + 1)
        g[0] = beta
        cs, sn = np.zeros(m), np.zeros(m)
        j = 0
        while j < m:
            Z.append(precond(V[j]))
            w = A_apply(Z[j])
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            hn = H[j + 1, j] = np.linalg.norm(w)
            V.append(w / hn if hn > 0.0 else w)
            for i in range(j):                       # earlier rotations
                a, c = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * a + sn[i] * c
                H[i + 1, j] = -sn[i] * a + cs[i] * c
            den = np.hypot(H[j, j], H[j + 1, j])      # new rotation
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j], H[j + 1, j] = den, 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            j += 1
            steps += 1
            hist.append(abs(g[j]))
            if hist[-1] <= rtol * bnorm or hn == 0.0:   # converged, or exact
                break
        y = sla.solve_triangular(H[:j, :j], g[:j])
        for i in range(j):
            x = x + y[i] * Z[i]
        r = b - A_apply(x)
        hist[-1] = np.linalg.norm(r)   # the true residual ends every cycle
        if hist[-1] <= rtol * bnorm:
            break
    return x, hist


def mg_solve(hier, b, rtol=1e-10, maxit=200, x0=None):
    """MG-preconditioned flexible CG on the finest level."""
    A = hier.A
    return fcg(lambda v: A @ v, hier.vcycle, b, rtol, maxit, x0)


def fractional_iterations(hist, digits=8):
    """nu = -digits * log10(rbar), rbar = (||r_n|| / ||r_0||)^(1/n) (Sec. 3.3)."""
    n = len(hist) - 1
    rbar = (hist[-1] / hist[0]) ** (1.0 / n)
    return -digits / np.log10(rbar)
