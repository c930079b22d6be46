"""Sampled vertex-patch checks for meshes too large for the assembled oracle
(test infrastructure; the arithmetic is the oracle's: element blocks, the
patch's principal block and a dense solve).

A colour pass of Algorithm 1 changes x only on the union of the Dirichlet
spaces V_j of that colour's patches, and on V_j by A_j^{-1} r_j with r_j the
patch's local residual evaluated at the x before the pass (patches of one
colour share no DoF and do not couple).  These helpers compute, for sampled
vertices, what the oracle's dense patch solve gives, and the mask of every DoF
that the colour may touch."""
import numpy as np
import scipy.linalg as sla

from oracle.assembly import block_apply, element_blocks, principal_block


def cell_id(dim, N, c):
    return int(sum(int(c[e]) * N ** e for e in range(dim)))


def local_nodes(dim, n):
    """(n^d, d) node multi-indices of a cell, direction 0 fastest."""
    idx = np.arange(n ** dim)
    return np.stack([(idx // n ** e) % n for e in range(dim)], axis=1)


def patch_cells_and_mask(dim, k, N, v, full=False):
    """Flat numbers of the 2^d cells of the patch at interior vertex v
    (ascending) and the boolean mask of the Dirichlet space V_j over their
    DoFs (patch-boundary nodes removed, except at ends on the domain
    boundary; full: every DoF of the patch cells, the full kernel's space)."""
    n = k + 1
    loc = local_nodes(dim, n)
    cells, mask = [], []
    for t in range(2 ** dim):
        o = [(t >> e) & 1 for e in range(dim)]
        cells.append(cell_id(dim, N, [v[e] - 1 + o[e] for e in range(dim)]))
        a = np.array(o)[None, :] * n + loc
        ok = np.ones(n ** dim, bool)
        if not full:
            for e in range(dim):
                ok &= (a[:, e] != 0) | (v[e] == 1)
                ok &= (a[:, e] != 2 * n - 1) | (v[e] == N - 1)
        mask.append(ok)
    return cells, np.concatenate(mask)


def sample_vertices(dim, N, colour, seed, count):
    """Vertices of one colour: both extreme vertices per direction (patches
    touching the domain boundary, first and last patch of the launch) and
    random ones."""
    rng = np.random.default_rng(seed)
    par = [(colour >> e) & 1 for e in range(dim)]
    choices = [np.arange(2 - p, N, 2) for p in par]   # v_e = p (mod 2), 1 <= v_e <= N-1
    out = {tuple(int(c[0]) for c in choices), tuple(int(c[-1]) for c in choices)}
    for e in range(dim):
        for end in (choices[e][0], choices[e][-1]):
            v = [int(rng.choice(choices[f])) for f in range(dim)]
            v[e] = int(end)
            out.add(tuple(v))
    total = int(np.prod([len(c) for c in choices]))
    while len(out) < min(count, total):
        out.add(tuple(int(rng.choice(c)) for c in choices))
    return sorted(out)


def colour_touch_mask(dim, k, N, colour, full=False):
    """Boolean mask over all DoFs: True where some patch of `colour` has the
    DoF in its Dirichlet space V_j (full: in one of its cells).  Along direction e a DoF of cell c_e, node
    i_e lies in the patch with vertex v_e = c_e (it is in the upper patch cell)
    or v_e = c_e + 1 (lower patch cell), whichever has the colour's parity."""
    n = k + 1
    nl = n ** dim
    cells = np.arange(N ** dim)
    loc = local_nodes(dim, n)
    ok = np.ones((N ** dim, nl), bool)
    for e in range(dim):
        ce = (cells // N ** e) % N
        p = (colour >> e) & 1
        v = np.where(ce % 2 == p, ce, ce + 1)               # the colour's vertex next to the cell
        upper = (v == ce)                                    # the cell is the patch's upper cell
        a = np.where(upper[:, None], n + loc[None, :, e], loc[None, :, e])
        inside = (v >= 1) & (v <= N - 1)
        good = ((a != 0) | (v[:, None] == 1)) & ((a != 2 * n - 1) | (v[:, None] == N - 1))
        ok &= inside[:, None] & (True if full else good)
    return ok.ravel()


class PatchOracle:
    """Dense patch solves of the oracle on an N^d mesh, factors cached per
    patch type (the patch matrix depends only on which ends touch the domain
    boundary)."""

    def __init__(self, dim, k, N, variant="consistent", kappa=1.0, eta=1.0):
        # variant "full": the full kernel (every patch DoF, the global residual)
        self.dim, self.k, self.N, self.variant = dim, k, N, variant
        self.blocks = element_blocks(dim, k, N, kappa, eta)
        self.no_last = element_blocks(dim, k, N, kappa, eta, part="no_last") if variant == "paper" else None
        self.cache = {}

    def _type(self, v):
        return tuple((v[e] == 1, v[e] == self.N - 1) for e in range(self.dim))

    def _factors(self, v, cells, mask):
        key = self._type(v)
        if key not in self.cache:
            D = principal_block(self.dim, self.k, self.N, self.blocks, cells)
            chol = sla.cho_factor(D[np.ix_(mask, mask)], lower=True)
            Abar = None
            if self.variant == "paper":
                Abar = principal_block(self.dim, self.k, self.N, self.blocks, cells, outer=self.no_last)[mask]
            self.cache[key] = (chol, Abar)
        return self.cache[key]

    def update(self, v, b, x0):
        """(global DoF indices of V_j, A_j^{-1} r_j) for the patch at vertex v,
        r_j the local residual at x0 (consistent and full: R_j (b - A x0);
        paper: R_j b - Abar_j Rbar_j x0, Sec. 3.1)."""
        n = self.k + 1
        nl = n ** self.dim
        cells, mask = patch_cells_and_mask(self.dim, self.k, self.N, v, full=self.variant == "full")
        dofs = np.concatenate([np.arange(nl) + c * nl for c in cells])
        chol, Abar = self._factors(v, cells, mask)
        if self.variant in ("consistent", "full"):
            Ax = block_apply(self.dim, self.k, self.N, self.blocks, x0, cells).ravel()[mask]
        else:
            Ax = Abar @ x0[dofs]
        r = b[dofs][mask] - Ax
        return dofs[mask], sla.cho_solve(chol, r)
