"""Pins of the oracle's multigrid pieces (Sec. 3) against properties the
paper and the mathematics fix."""
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle.assembly import assemble, mass_matrix_cell
from oracle.basis import gauss_lobatto
from oracle.direct import GlobalFD, one_d_matrices
from oracle.layout import node_coordinates
from oracle.mg import (Hierarchy, Level, fcg, fractional_iterations, mg_solve,
                       prolongation, smooth, vertex_patches)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ transfer
@pytest.mark.parametrize("dim,k,Nc", [(1, 3, 2), (2, 2, 2), (2, 3, 4), (3, 2, 2)])
def test_prolongation_reproduces_polynomials(dim, k, Nc):
    # canonical embedding (Sec. 3): a polynomial of degree <= k per direction
    # on the coarse mesh is the same function on the fine mesh
    rng = np.random.default_rng(3)
    coeff = rng.standard_normal((k + 1,) * dim)

    def poly(p):
        val = np.zeros(len(p))
        for idx in np.ndindex(*coeff.shape):
            val += coeff[idx] * np.prod([p[:, e] ** idx[e] for e in range(dim)], axis=0)
        return val

    nodes = gauss_lobatto(k)[0]
    P = prolongation(dim, k, Nc)
    xc = poly(node_coordinates(dim, Nc, nodes))
    xf = poly(node_coordinates(dim, 2 * Nc, nodes))
    assert np.max(np.abs(P @ xc - xf)) < 1e-12 * np.max(np.abs(xf))


@pytest.mark.parametrize("dim,k,Nc", [(1, 2, 2), (2, 2, 2), (2, 3, 4), (3, 2, 2)])
def test_galerkin_identity_with_doubled_penalty(dim, k, Nc):
    # The embedded coarse functions are continuous across the new fine faces
    # and every coarse face is covered by fine faces with twice the penalty
    # (gamma ~ 1/h): P^T A_fine(eta) P = A_coarse(2 eta) exactly.
    P = prolongation(dim, k, Nc)
    Af = assemble(dim, k, 2 * Nc, kappa=1.2, eta=1.0)
    Ac = assemble(dim, k, Nc, kappa=1.2, eta=2.0).toarray()
    G = (P.T @ Af @ P).toarray()
    assert np.max(np.abs(G - Ac)) < 1e-12 * np.max(np.abs(Ac))


@pytest.mark.parametrize("dim,k,Nc", [(2, 3, 2), (3, 2, 2)])
def test_mass_is_preserved_by_embedding(dim, k, Nc):
    P = prolongation(dim, k, Nc)
    Mf = np.kron(np.eye((2 * Nc) ** dim), mass_matrix_cell(dim, k, 2 * Nc))
    Mc = np.kron(np.eye(Nc ** dim), mass_matrix_cell(dim, k, Nc))
    assert np.max(np.abs(P.T.toarray() @ Mf @ P.toarray() - Mc)) < 1e-14


# ------------------------------------------------------------------ patches
@pytest.mark.parametrize("dim,k,N", [(2, 2, 4), (2, 3, 5), (3, 2, 4), (2, 1, 2)])
def test_patch_structure(dim, k, N):
    n = k + 1
    pats = vertex_patches(dim, k, N)
    assert len(pats) == (N - 1) ** dim
    for p in pats:
        sizes = []
        for (lb, rb) in p["type"]:
            sizes.append(2 * k + int(lb) + int(rb))
        assert len(p["V"]) == np.prod(sizes)
        assert len(p["dofs"]) == (2 * n) ** dim
    # same-colour patches cover disjoint cells
    for c in range(2 ** dim):
        mem = [p["dofs"] for p in pats if p["colour"] == c]
        if not mem:
            continue
        cells = np.concatenate(mem)
        assert len(np.unique(cells)) == len(cells)
    # every DoF is in some V_j (boundary ends kept): nothing is left unsmoothed
    allV = np.unique(np.concatenate([p["V"] for p in pats]))
    assert len(allV) == N ** dim * n ** dim


@pytest.mark.parametrize("dim,k,N", [(2, 2, 6), (3, 2, 4)])
def test_same_colour_patches_do_not_couple(dim, k, N):
    A = assemble(dim, k, N).tocsr()
    pats = vertex_patches(dim, k, N)
    for c in range(2 ** dim):
        mem = [p for p in pats if p["colour"] == c]
        for i in range(len(mem)):
            for j in range(len(mem)):
                if i != j:
                    blk = A[mem[i]["V"]][:, mem[j]["V"]]
                    assert blk.nnz == 0 or np.abs(blk.data).max() == 0.0


@pytest.mark.parametrize("dim,k,N", [(2, 2, 8), (3, 2, 4)])
def test_colour_pass_independent_of_patch_order(dim, k, N):
    lev = Level(dim, k, N)
    rng = np.random.default_rng(5)
    b = rng.standard_normal(lev.ndof)
    x0 = rng.standard_normal(lev.ndof)
    ref = smooth(lev, x0, b)
    perm_rng = np.random.default_rng(6)
    other = smooth(lev, x0, b, patch_order=lambda c, m: perm_rng.permutation(m))
    assert np.array_equal(ref, other)


@pytest.mark.parametrize("dim,k,N", [(2, 3, 4), (3, 2, 4)])
def test_local_solve_zeroes_local_residual(dim, k, N):
    lev = Level(dim, k, N)
    rng = np.random.default_rng(7)
    b = rng.standard_normal(lev.ndof)
    x = rng.standard_normal(lev.ndof)
    for p in lev.patches[:: max(1, len(lev.patches) // 5)]:
        r = b[p["V"]] - lev.A[p["V"]] @ x
        x2 = x.copy()
        x2[p["V"]] += sla.cho_solve(p["chol"], r)
        r2 = b[p["V"]] - lev.A[p["V"]] @ x2
        assert np.linalg.norm(r2) < 1e-12 * np.linalg.norm(r)


def _patch_1d(k, N, v, kappa=1.0, eta=1.0):
    """Restriction of the global 1D L, M to the 1D index set of patch v."""
    L, M = one_d_matrices(k, N, kappa, eta)
    n = k + 1
    start = (v - 1) * n
    idx = np.arange(start, start + 2 * n)
    keep = np.ones(2 * n, dtype=bool)
    if v != 1:
        keep[0] = False
    if v != N - 1:
        keep[-1] = False
    idx = idx[keep]
    return L[np.ix_(idx, idx)], M[np.ix_(idx, idx)]


@pytest.mark.parametrize("dim,k,N", [(2, 2, 4), (2, 3, 6), (3, 2, 4), (3, 3, 4)])
def test_fast_diagonalisation_equals_dense_inverse(dim, k, N):
    # Eqs. inverse2d / inverse3d / fast_inverse: A_j^{-1} = (x)S (sum Lambda)^{-1} (x)S^T
    lev = Level(dim, k, N, kappa=1.1, eta=1.0)
    for p in lev.patches:
        v = p["vertex"]
        Ls, Ms = zip(*[_patch_1d(k, N, v[e], 1.1) for e in range(dim)])
        Ss, lams = [], []
        for e in range(dim):
            lam, S = sla.eigh(Ls[e], Ms[e])
            assert np.allclose(S.T @ Ms[e] @ S, np.eye(len(lam)), atol=1e-12)
            assert np.allclose(Ls[e] @ S, Ms[e] @ S * lam[None, :], atol=1e-9 * np.abs(Ls[e]).max())
            Ss.append(S)
            lams.append(lam)
        # tensor in slot order d-1 ... 0 (slot 0 fastest)
        Skron = np.ones((1, 1))
        D = np.zeros(1)
        for e in reversed(range(dim)):
            Skron = np.kron(Skron, Ss[e])
            D = (D[:, None] + lams[e][None, :]).ravel()
        inv_fd = Skron @ np.diag(1.0 / D) @ Skron.T
        # dense A_j in the same (patch-lexicographic) order
        Aj = lev.A[p["V"]][:, p["V"]].toarray()
        # map patch-lexicographic order to the oracle's sorted global order
        order = _patch_lex_to_global(dim, k, N, v)
        pos = np.searchsorted(p["V"], order)
        Aj_lex = Aj[np.ix_(pos, pos)]
        inv_dense = np.linalg.inv(Aj_lex)
        assert np.max(np.abs(inv_fd - inv_dense)) < 1e-12 * np.max(np.abs(inv_dense))


def _patch_lex_to_global(dim, k, N, v):
    n = k + 1
    ranges = []
    for e in range(dim):
        a = np.arange(2 * n)
        keep = np.ones(2 * n, dtype=bool)
        if v[e] != 1:
            keep[0] = False
        if v[e] != N - 1:
            keep[-1] = False
        ranges.append(a[keep])
    grids = np.meshgrid(*ranges[::-1], indexing="ij")      # slot d-1 slowest
    coords = np.stack([g.ravel() for g in grids[::-1]], axis=1)  # (m, d) slot 0 fastest
    cells = np.array(v)[None, :] - 1 + coords // n
    local = coords % n
    c = np.zeros(len(coords), dtype=np.int64)
    loc = np.zeros(len(coords), dtype=np.int64)
    s1 = s2 = 1
    for e in range(dim):
        c += cells[:, e] * s1
        loc += local[:, e] * s2
        s1 *= N
        s2 *= n
    return c * n ** dim + loc


# ------------------------------------------------------------------ V-cycle / solver
@pytest.mark.parametrize("variant", ["consistent", "full", "clamped"])
@pytest.mark.parametrize("dim,k,N,L", [(2, 2, 8, 3), (3, 2, 4, 2)])
def test_vcycle_is_symmetric(dim, k, N, L, variant):
    # multiplicative over colours with the colours reversed in post-smoothing
    # and exact local solves: a symmetric preconditioner for CG (for every
    # kernel whose residual is exact; the paper's Dirichlet residual is not)
    H = Hierarchy(dim, k, N, L, variant=variant)
    rng = np.random.default_rng(8)
    x = rng.standard_normal(H.A.shape[0])
    y = rng.standard_normal(H.A.shape[0])
    a = H.vcycle(x) @ y
    b = x @ H.vcycle(y)
    assert abs(a - b) < 1e-13 * max(abs(a), 1.0) * 10


def test_paper_residual_vcycle_is_not_symmetric():
    # the Dirichlet kernel's inconsistent residual breaks the symmetry, which
    # is why the paper's setting runs GMRES
    H = Hierarchy(3, 2, 4, 2, variant="paper")
    rng = np.random.default_rng(8)
    x = rng.standard_normal(H.A.shape[0])
    y = rng.standard_normal(H.A.shape[0])
    a = H.vcycle(x) @ y
    b = x @ H.vcycle(y)
    assert abs(a - b) > 1e-6 * abs(a)


def test_one_level_fcg_converges_in_one_iteration():
    H = Hierarchy(2, 3, 2, 1)
    rng = np.random.default_rng(9)
    b = rng.standard_normal(H.A.shape[0])
    x, hist = mg_solve(H, b, rtol=1e-12)
    assert len(hist) == 2


@pytest.mark.parametrize("dim,k,N,L", [(2, 1, 4, 2), (2, 2, 4, 2), (2, 3, 8, 3), (3, 1, 4, 2), (3, 2, 4, 2), (3, 3, 2, 1)])
def test_tiny_mesh_mg_equals_direct(dim, k, N, L):
    H = Hierarchy(dim, k, N, L, kappa=0.8)
    rng = np.random.default_rng(10)
    b = rng.standard_normal(H.A.shape[0])
    x, hist = mg_solve(H, b, rtol=1e-13)
    xd = np.linalg.solve(H.A.toarray(), b)
    xf = GlobalFD(dim, k, N, kappa=0.8).solve(b)
    scale = np.abs(xd).max()
    assert np.abs(xf - xd).max() < 1e-12 * scale
    assert np.abs(x - xd).max() < 1e-10 * scale


def test_fcg_equals_pcg_for_fixed_spd_preconditioner():
    # flexible CG reduces to PCG (same iterates) for a fixed SPD B; compare
    # with a textbook PCG written out here
    rng = np.random.default_rng(11)
    n = 60
    Q = rng.standard_normal((n, n))
    A = Q @ Q.T + n * np.eye(n)
    Bm = np.diag(1.0 / np.diag(A))
    b = rng.standard_normal(n)
    x, hist = fcg(lambda v: A @ v, lambda v: Bm @ v, b, rtol=1e-12)
    xr = np.zeros(n)
    r = b.copy()
    z = Bm @ r
    p = z.copy()
    href = [np.linalg.norm(r)]
    for _ in range(len(hist) - 1):
        q = A @ p
        a = (r @ z) / (p @ q)
        xr += a * p
        rn = r - a * q
        href.append(np.linalg.norm(rn))
        zn = Bm @ rn
        beta = (rn @ zn) / (r @ z)
        p = zn + beta * p
        r, z = rn, zn
    assert np.allclose(hist, href, rtol=1e-9)
    assert np.allclose(x, xr, rtol=1e-9, atol=1e-12)


def test_fractional_iteration_count():
    # one decade per iteration -> 8 iterations for 8 decades; four -> 2
    assert abs(fractional_iterations([1.0, 0.1, 0.01]) - 8.0) < 1e-12
    assert abs(fractional_iterations([1.0, 1e-4, 1e-8]) - 2.0) < 1e-12


def test_nu_bounded_and_near_table2():
    # Table 2 (Dirichlet kernel, 3D): nu between 4.4 and 6.5.  The oracle uses
    # FCG and the consistent residual, so only the ballpark is compared: nu
    # within a factor 2 of the table for Q2..Q3 on L = 2, 3 and not growing
    # with the level.
    ref = np.loadtxt(os.path.join(GOLDEN, "table2_dirichlet_nu.txt"))
    nus = []
    for N, L in ((4, 2), (8, 3)):
        H = Hierarchy(3, 3, N, L)
        b = np.ones(H.A.shape[0])
        from oracle.assembly import rhs_from_nodal
        b = rhs_from_nodal(3, 3, N, b)
        _, hist = mg_solve(H, b, rtol=1e-8)
        nus.append(fractional_iterations(hist))
    q3 = ref[:2, 1]
    for nu, r in zip(nus, q3):
        assert r / 2 <= nu <= 2 * r
    assert nus[1] < nus[0] * 1.5


# --------------------------------------------------------------------- GMRES
def _krylov_min_residual(Aop, b, j):
    """Brute force: min over y in K_j(Aop, b) of ||b - Aop y||_2, with the
    Krylov vectors normalised one by one and orthonormalised by QR."""
    cols, v = [], b / np.linalg.norm(b)
    for _ in range(j):
        cols.append(v)
        v = Aop @ v
        v = v / np.linalg.norm(v)
    Q, _ = np.linalg.qr(np.column_stack(cols))
    y = np.linalg.lstsq(Aop @ Q, b, rcond=None)[0]
    return np.linalg.norm(b - Aop @ (Q @ y))


def test_gmres_history_is_the_krylov_minimum():
    # GMRES (Sec. 3.3's outer solver) minimises ||b - A x|| over x in
    # K_j(A B, b) mapped by B: with right preconditioning its history equals
    # the brute-force minimum over the Krylov space of A B, for a fixed B
    from oracle.mg import gmres
    rng = np.random.default_rng(21)
    n = 30
    A = 4.0 * np.eye(n) + 0.6 * rng.standard_normal((n, n))        # nonsymmetric
    Bm = np.linalg.inv(A + 0.8 * rng.standard_normal((n, n)) / np.sqrt(n))
    b = rng.standard_normal(n)
    for Bop in (np.eye(n), Bm):
        x, hist = gmres(lambda v: A @ v, lambda v: Bop @ v, b, rtol=1e-12, maxit=n, restart=n)
        assert hist[0] == pytest.approx(np.linalg.norm(b))
        for j in range(1, min(len(hist), 12)):
            assert abs(hist[j] - _krylov_min_residual(A @ Bop, b, j)) <= 1e-9 * np.linalg.norm(b)
        assert np.linalg.norm(b - A @ x) <= 1e-11 * np.linalg.norm(b)
        assert np.allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-10 * np.abs(np.linalg.solve(A, b)).max())


def test_left_gmres_history_is_the_preconditioned_krylov_minimum():
    # GMRES preconditioned from the left minimises ||B (b - A x)|| over x in
    # the Krylov space K_j(B A, B b): its history equals that brute-force
    # minimum (a different norm from the right-preconditioned one)
    from oracle.mg import gmres
    rng = np.random.default_rng(23)
    n = 30
    A = 4.0 * np.eye(n) + 0.6 * rng.standard_normal((n, n))
    Bm = np.linalg.inv(A + 0.8 * rng.standard_normal((n, n)) / np.sqrt(n))
    b = rng.standard_normal(n)
    x, hist = gmres(lambda v: A @ v, lambda v: Bm @ v, b, rtol=1e-12, maxit=n, restart=n, side="left")
    assert hist[0] == pytest.approx(np.linalg.norm(Bm @ b))
    # (B A is close to the identity here, so the residual falls fast; the
    # brute-force Krylov basis is compared while it is well conditioned)
    checked = 0
    for j in range(1, len(hist)):
        if hist[j] < 1e-4 * hist[0]:
            break
        assert abs(hist[j] - _krylov_min_residual(Bm @ A, Bm @ b, j)) <= 1e-9 * np.linalg.norm(Bm @ b)
        checked += 1
    assert checked >= 4
    assert np.allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-9 * np.abs(np.linalg.solve(A, b)).max())
    _, right = gmres(lambda v: A @ v, lambda v: Bm @ v, b, rtol=1e-12, maxit=n, restart=n)
    assert abs(hist[3] - right[3]) > 1e-6 * hist[0]      # not the right-preconditioned history


def test_gmres_restarts_and_converges():
    from oracle.mg import gmres
    rng = np.random.default_rng(22)
    n = 60
    A = 3.0 * np.eye(n) + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    x, hist = gmres(lambda v: A @ v, lambda v: v, b, rtol=1e-10, maxit=200, restart=5)
    assert all(h1 <= h0 * (1 + 1e-12) for h0, h1 in zip(hist, hist[1:]))
    assert len(hist) - 1 > 5                       # needed at least one restart
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b)
    # restart 5 minimises over 5 steps only: its first cycle equals full GMRES
    _, full = gmres(lambda v: A @ v, lambda v: v, b, rtol=1e-10, maxit=200, restart=200)
    assert np.allclose(hist[:5], full[:5], rtol=1e-10)


# ------------------------------------------------------ paper Dirichlet kernel
@pytest.mark.parametrize("dim,k,N", [(2, 2, 4), (2, 3, 4), (3, 2, 4)])
def test_dirichlet_kernel_residual_exact_for_continuous_x(dim, k, N):
    # Sec. 3.1: the Dirichlet kernel's residual misses only the last face
    # term -[[u]].{grad v} on the patch-boundary faces.  That term vanishes
    # when u has no jump there, so for a continuous u the paper's residual is
    # the exact one; for a discontinuous u it is not.
    cons = Level(dim, k, N, variant="consistent")
    pap = Level(dim, k, N, variant="paper")
    nodes, _ = gauss_lobatto(k)
    X = node_coordinates(dim, N, nodes)
    u_cont = np.prod(np.cos(1.3 * X + 0.4), axis=1) + X[:, 0] ** 2  # continuous (GLL traces agree)
    rng = np.random.default_rng(5)
    b = rng.standard_normal(cons.ndof)
    u_disc = rng.standard_normal(cons.ndof)
    from oracle.mg import local_residual
    worst_cont, worst_disc = 0.0, np.inf
    for pc, pp in zip(cons.patches, pap.patches):
        assert np.array_equal(pc["V"], pp["V"])
        rc = local_residual(pc, b, u_cont)
        rp = local_residual(pp, b, u_cont)
        worst_cont = max(worst_cont, np.abs(rc - rp).max() / np.abs(rc).max())
        d = np.abs(local_residual(pc, b, u_disc) - local_residual(pp, b, u_disc)).max()
        worst_disc = min(worst_disc, d / np.abs(local_residual(pc, b, u_disc)).max())
    assert worst_cont <= 1e-12
    assert worst_disc > 1e-3          # every patch sees the dropped term


def test_gmres_dirichlet_kernel_reproduces_table2():
    # Table 2, Dirichlet kernel: 3D, f = 1, GMRES to 1e-8 preconditioned by
    # the V-cycle with the paper's (inconsistent) Dirichlet-kernel residual.
    # The oracle reproduces the printed nu within 20 % at L = 2 (Q3, Q4) and
    # L = 3 (Q3), and nu does not grow with L.  (Keeping the patch-side half
    # of the dropped face term instead gives nu near 10 at L = 2 and 18 at
    # L = 3.)
    from oracle.assembly import rhs_from_nodal
    from oracle.mg import gmres
    ref = np.loadtxt(os.path.join(GOLDEN, "table2_dirichlet_nu.txt"))
    got = {}
    for k, L in ((3, 2), (3, 3), (4, 2)):
        N = 1 << L
        H = Hierarchy(3, k, N, L, variant="paper")
        b = rhs_from_nodal(3, k, N, np.ones(H.A.shape[0]))
        _, hist = gmres(lambda v: H.A @ v, H.vcycle, b, rtol=1e-8, maxit=60)
        got[(k, L)] = fractional_iterations(hist)
        printed = ref[L - 2, k - 2]
        assert abs(got[(k, L)] - printed) <= 0.2 * printed, (k, L, got[(k, L)], printed)
    assert got[(3, 3)] <= 1.2 * got[(3, 2)]
    # Table 4's single-GPU column prints the same Q3 setting with other values
    # (5.3, 6.2 at L = 2, 3): the oracle lies within 10 % of those
    ref4 = np.loadtxt(os.path.join(GOLDEN, "table4_local_nu.txt"))
    for L in (2, 3):
        assert abs(got[(3, L)] - ref4[L - 2, 1]) <= 0.1 * ref4[L - 2, 1], (L, got[(3, L)])


# ---------------------------------------------------------------- full kernel
@pytest.mark.parametrize("dim,k", [(2, 2), (2, 3), (3, 2)])
def test_full_kernel_is_exact_on_a_one_patch_mesh(dim, k):
    # N = 2: one interior vertex whose patch is the whole mesh, so the full
    # kernel's local space is everything and one smoothing step solves Ax = b
    lev = Level(dim, k, 2, variant="full")
    assert len(lev.patches) == 1 and len(lev.patches[0]["V"]) == lev.ndof
    b = np.random.default_rng(3).standard_normal(lev.ndof)
    x = smooth(lev, np.zeros(lev.ndof), b)
    assert np.allclose(x, np.linalg.solve(lev.A.toarray(), b), rtol=0, atol=1e-11 * np.abs(x).max())


@pytest.mark.parametrize("dim,k,N", [(2, 3, 4), (3, 2, 4)])
def test_full_kernel_patch_matrix_is_a_kronecker_sum(dim, k, N):
    # A_j over all 2n nodes per direction = sum_d (x) (L_patch in d, M_patch
    # elsewhere) with L_patch, M_patch the global 1D matrices restricted to
    # the patch's 2n nodes (Sec. 2.2 on the patch), and its fast
    # diagonalisation (Eq. fast_inverse) inverts it
    lev = Level(dim, k, N, variant="full")
    L1, M1 = one_d_matrices(k, N)
    n = k + 1
    for p in lev.patches[:: max(1, len(lev.patches) // 4)]:
        v = p["vertex"]
        mats = []
        for e in range(dim):
            idx = np.arange((v[e] - 1) * n, (v[e] + 1) * n)
            mats.append((L1[np.ix_(idx, idx)], M1[np.ix_(idx, idx)]))
        # patch-local lexicographic order (direction 0 fastest) -> global
        loc = np.zeros((2 * n,) * dim, dtype=np.int64)
        for a in np.ndindex(*(2 * n,) * dim):
            cell = [v[e] - 1 + a[e] // n for e in range(dim)]
            node = [a[e] % n for e in range(dim)]
            cf = sum(cell[e] * N ** e for e in range(dim))
            nf = sum(node[e] * n ** e for e in range(dim))
            loc[a] = cf * n ** dim + nf
        order = loc.transpose(*range(dim)[::-1]).ravel()     # direction 0 fastest
        Aj = lev.A[order][:, order].toarray()
        K = np.zeros_like(Aj)
        for d in range(dim):
            term = np.ones((1, 1))
            for e in range(dim - 1, -1, -1):
                term = np.kron(term, mats[e][0] if e == d else mats[e][1])
            K += term
        assert np.abs(Aj - K).max() <= 1e-12 * np.abs(Aj).max()
        lam_S = [sla.eigh(Le, Me) for Le, Me in mats]
        lam = sum(np.meshgrid(*[ls[0] for ls in lam_S[::-1]], indexing="ij")[::-1][d] for d in range(dim))
        S = np.ones((1, 1))
        for e in range(dim - 1, -1, -1):
            S = np.kron(S, lam_S[e][1])
        inv = S @ np.diag(1.0 / lam.ravel()) @ S.T
        assert np.abs(inv @ Aj - np.eye(len(Aj))).max() < 1e-9


def test_gmres_full_kernel_near_table1():
    # Table 1 (full kernel) against Table 2 (Dirichlet kernel): the full kernel
    # needs fewer iterations, and nu does not grow with L.  The oracle's nu
    # lies 25-40 % below the printed values (Q3: 2.25 / 2.34 at L = 2 / 3
    # against 3.4 / 3.7), so the table itself is matched to a factor 1.6 only.
    from oracle.assembly import rhs_from_nodal
    from oracle.mg import gmres
    ref1 = np.loadtxt(os.path.join(GOLDEN, "table1_full_nu.txt"))
    got = {}
    for L in (2, 3):
        N = 1 << L
        nu = {}
        for variant in ("full", "paper"):
            H = Hierarchy(3, 3, N, L, variant=variant)
            b = rhs_from_nodal(3, 3, N, np.ones(H.A.shape[0]))
            _, hist = gmres(lambda v: H.A @ v, H.vcycle, b, rtol=1e-8, maxit=60)
            nu[variant] = fractional_iterations(hist)
        printed = ref1[L - 2, 1]
        assert printed / 1.6 <= nu["full"] <= printed * 1.6, (L, nu, printed)
        assert nu["full"] < nu["paper"]
        got[L] = nu["full"]
    assert got[3] <= 1.2 * got[2]


@pytest.mark.parametrize("dim,k,N", [(2, 2, 4), (2, 3, 8), (3, 1, 4)])
def test_full_kernel_colour_pass_is_block_jacobi(dim, k, N):
    # the residual is updated once per colour ("globally", Sec. 3.1), so one
    # colour pass is a block-Jacobi step over the colour's patches: solve
    # with A on the union of their DoFs after deleting the couplings between
    # different patches (they share faces, not DoFs), add, leave the rest
    lev = Level(dim, k, N, variant="full")
    rng = np.random.default_rng(9)
    b = rng.standard_normal(lev.ndof)
    x0 = rng.standard_normal(lev.ndof)
    A = lev.A.toarray()
    r = b - A @ x0
    for c in range(2 ** dim):
        owner = -np.ones(lev.ndof, dtype=np.int64)
        for i, p in enumerate(lev.patches):
            if p["colour"] == c:
                assert np.all(owner[p["V"]] < 0)
                owner[p["V"]] = i
        U = np.flatnonzero(owner >= 0)
        D = A[np.ix_(U, U)] * (owner[U][:, None] == owner[U][None, :])
        expect = x0.copy()
        expect[U] += np.linalg.solve(D, r[U])
        got = smooth(lev, x0, b, colours=[c])
        assert np.allclose(got, expect, rtol=0, atol=1e-10 * np.abs(expect).max())


# ------------------------------------------------------------- clamped kernel
@pytest.mark.parametrize("dim,k,N", [(2, 2, 4), (2, 3, 6), (3, 2, 4), (3, 3, 4)])
def test_clamped_residual_needs_only_the_patch_cells(dim, k, N):
    # Sec. 3.1: for v with v = 0 and grad v . n = 0 on the patch boundary all
    # face terms there vanish, so B^T R_D (b - A x) does not see x outside the
    # patch cells (a space without the derivative condition would); the
    # clamped space has (2k-2)^d functions for an interior patch
    lev = Level(dim, k, N, variant="clamped")
    rng = np.random.default_rng(31)
    b = rng.standard_normal(lev.ndof)
    x = rng.standard_normal(lev.ndof)
    for p in lev.patches:
        interior = all(1 < p["vertex"][e] < N - 1 for e in range(dim))
        if interior:
            assert p["B"].shape[1] == (2 * k - 2) ** dim
        inside = np.zeros(lev.ndof, dtype=bool)
        inside[p["dofs"]] = True
        x2 = x + np.where(inside, 0.0, rng.standard_normal(lev.ndof))
        r1 = p["B"].T @ (b - lev.A @ x)[p["dofs"]]
        r2 = p["B"].T @ (b - lev.A @ x2)[p["dofs"]]
        assert np.abs(r1 - r2).max() <= 1e-12 * np.abs(r1).max()
    # the Dirichlet space without the derivative condition does see outside
    pd = Level(dim, k, N, variant="consistent").patches[0]
    inside = np.zeros(lev.ndof, dtype=bool)
    inside[pd["dofs"]] = True
    x2 = x + np.where(inside, 0.0, 1.0)
    assert np.abs((lev.A @ (x - x2))[pd["V"]]).max() > 1e-3


@pytest.mark.parametrize("dim,k,N", [(2, 3, 4), (3, 2, 4)])
def test_clamped_local_solve_and_order(dim, k, N):
    lev = Level(dim, k, N, variant="clamped")
    rng = np.random.default_rng(32)
    b = rng.standard_normal(lev.ndof)
    x0 = rng.standard_normal(lev.ndof)
    for p in lev.patches[:: max(1, len(lev.patches) // 5)]:
        x = smooth(lev, x0, b, colours=[p["colour"]])
        # after its colour pass a patch's residual vanishes on its clamped space
        r = p["B"].T @ (b - lev.A @ x)[p["dofs"]]
        assert np.abs(r).max() <= 1e-10 * np.abs(p["B"].T @ (b - lev.A @ x0)[p["dofs"]]).max()
    perm_rng = np.random.default_rng(4)
    ref = smooth(lev, x0, b)
    other = smooth(lev, x0, b, patch_order=lambda c, m: perm_rng.permutation(m))
    assert np.allclose(ref, other, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_gmres_clamped_kernel_reproduces_table2():
    # Table 2, clamped kernel, read with GMRES preconditioned from the left
    # (its residual, and so nu, measured after the V-cycle): within 20 % of
    # the printed values for Q3 at L = 3 and Q5 at L = 2, within 40 % for Q3
    # at L = 2 (the 4^3 mesh, where 26 of the 27 patches touch the domain
    # boundary), nu level-independent as printed.  Preconditioned from the
    # right (the Euclidean residual) the same V-cycle gives nu 1.7-1.9 times
    # the printed values and growing with L; writing the system in a
    # Hermite-type basis (value and derivative at the cell ends) moves nu by
    # only ~15 % -- neither explains the column.
    from oracle.assembly import rhs_from_nodal
    from oracle.mg import gmres
    ref = np.loadtxt(os.path.join(GOLDEN, "table2_clamped_nu.txt"))
    dirichlet = np.loadtxt(os.path.join(GOLDEN, "table2_dirichlet_nu.txt"))
    nus = {}
    for k, N, L, tol in ((3, 8, 3, 0.2), (5, 4, 2, 0.2), (3, 4, 2, 0.4)):
        H = Hierarchy(3, k, N, L, variant="clamped")
        b = rhs_from_nodal(3, k, N, np.ones(H.A.shape[0]))
        _, hist = gmres(lambda v: H.A @ v, H.vcycle, b, rtol=1e-8, maxit=100, side="left")
        nus[(k, L)] = fractional_iterations(hist)
        printed = ref[L - 2, k - 2]
        assert abs(nus[(k, L)] - printed) <= tol * printed, (k, L, nus[(k, L)], printed)
        assert nus[(k, L)] > dirichlet[L - 2, k - 2]      # the paper's ordering
    assert nus[(5, 2)] < nus[(3, 2)]                      # falls with the degree
    assert abs(nus[(3, 3)] - nus[(3, 2)]) < 0.2 * nus[(3, 2)]   # no growth with L


def test_clamped_space_closed_form_for_q2():
    # k = 2, interior patch: on the low cell a quadratic with v = v' = 0 at
    # its low end is a multiple of x^2, on the high cell one with v = v' = 0
    # at its high end is a multiple of (1 - x)^2; in the Gauss-Lobatto
    # Lagrange coefficients (nodes 0, 1/2, 1) these are (0, 1/4, 1) and
    # (1, 1/4, 0).  With a domain-boundary end the space gains that end's
    # value and derivative (2k and 2k + 2 functions).
    from oracle.mg import clamped_basis_1d
    B = clamped_basis_1d(2, False, False)
    expect = np.array([[0, 0.25, 1, 0, 0, 0], [0, 0, 0, 1, 0.25, 0]], dtype=float).T
    assert B.shape == (6, 2)
    proj = B @ (B.T @ expect)                      # expect lies in span(B)
    assert np.abs(proj - expect).max() < 1e-13
    assert np.allclose(B.T @ B, np.eye(2), atol=1e-13)
    for k in range(2, 8):
        assert clamped_basis_1d(k, False, False).shape[1] == 2 * k - 2
        assert clamped_basis_1d(k, True, False).shape[1] == 2 * k
        assert clamped_basis_1d(k, False, True).shape[1] == 2 * k
        assert clamped_basis_1d(k, True, True).shape[1] == 2 * k + 2


def test_full_kernel_at_most_three_steps_for_degree_four():
    # Sec. 3.3 on Table 1: for degrees 4 and higher the full kernel converges
    # (GMRES to 1e-8, f = 1) in at most three steps
    from oracle.assembly import rhs_from_nodal
    from oracle.mg import gmres
    for k in (4, 5):
        H = Hierarchy(3, k, 4, 2, variant="full")
        b = rhs_from_nodal(3, k, 4, np.ones(H.A.shape[0]))
        _, hist = gmres(lambda v: H.A @ v, H.vcycle, b, rtol=1e-8, maxit=10)
        assert len(hist) - 1 <= 3 and hist[-1] <= 1e-8 * hist[0], (k, hist)


def test_local_space_dimensions_for_q3():
    # Sec. 3.3: for Q3 the local space of an interior patch has 8^3 functions
    # for the full kernel, 6^3 for the Dirichlet kernel, 4^3 for the clamped
    N = 6
    interior = lambda p: all(1 < p["vertex"][e] < N - 1 for e in range(3))
    for variant, dim_vj in (("full", 8 ** 3), ("consistent", 6 ** 3), ("clamped", 4 ** 3)):
        lev = Level(3, 3, N, variant=variant)
        p = next(p for p in lev.patches if interior(p))
        size = p["B"].shape[1] if p["B"] is not None else len(p["V"])
        assert size == dim_vj, (variant, size)
