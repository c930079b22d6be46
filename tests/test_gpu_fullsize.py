"""Parity at the benchmark's full size (3D SIPG, 64^3 cells, Q3, 6 levels,
16.8M DoFs) in the launch configuration bench.py times (CUDA graphs on):
sampled outputs the oracle computes one by one (operator rows of sampled
cells; local solves of sampled vertex patches, interior and boundary), a
property that holds at any size (V-cycle symmetry), and whole solves against
the oracle's exact global fast-diagonalisation solve."""
import numpy as np
import pytest

from gpu_helpers import dev, gpu_available, host, make, rel_inf

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

from oracle.assembly import block_apply, element_blocks, principal_block, rhs_from_nodal  # noqa: E402
from oracle.basis import gauss_lobatto  # noqa: E402
from oracle.direct import GlobalFD  # noqa: E402
from oracle.layout import node_coordinates  # noqa: E402
from paper_2405_18982_gb300 import SIPG_FP32, SIPG_FP64, inputs  # noqa: E402

DIM, K, L2, NL = 3, 3, 6, 6
N = 1 << L2
n = K + 1
NLOC = n ** DIM


@pytest.fixture(scope="module")
def blocks():
    return element_blocks(DIM, K, N)


@pytest.fixture(scope="module")
def solvers():
    return {SIPG_FP64: make(DIM, K, L2, NL, prec=SIPG_FP64, graphs=1),
            SIPG_FP32: make(DIM, K, L2, NL, prec=SIPG_FP32, graphs=1)}


def _cell_id(c):
    return int(c[0] + N * (c[1] + N * c[2]))


def sample_cells(seed, count=600):
    rng = np.random.default_rng(seed)
    fixed = [(0, 0, 0), (N - 1, N - 1, N - 1), (0, N // 2, N - 1), (N // 2, 0, 5), (7, N - 1, 0)]
    cells = [_cell_id(c) for c in fixed] + list(rng.choice(N ** DIM, size=count, replace=False))
    return np.array(sorted(set(cells)))


def sample_patches(colour, seed, count=40):
    """Vertices of the given colour: boundary ones (v_e = 1 or N-1) and random."""
    rng = np.random.default_rng(seed)
    par = [(colour >> e) & 1 for e in range(DIM)]
    choices = [np.arange(1 + (1 - p), N, 2) for p in par]   # v_e of parity p, 1..N-1
    out = set()
    for e in range(DIM):
        for end in (choices[e][0], choices[e][-1]):
            v = [int(rng.choice(choices[f])) for f in range(DIM)]
            v[e] = int(end)
            out.add(tuple(v))
    out.add(tuple(int(c[0]) for c in choices))
    out.add(tuple(int(c[-1]) for c in choices))
    while len(out) < count:
        out.add(tuple(int(rng.choice(c)) for c in choices))
    return sorted(out)


def patch_cells_and_mask(v):
    cells, mask = [], []
    loc = np.array([[i % n, (i // n) % n, i // (n * n)] for i in range(NLOC)])
    for o in [(a, b, c) for c in (0, 1) for b in (0, 1) for a in (0, 1)]:
        cells.append(_cell_id([v[e] - 1 + o[e] for e in range(DIM)]))
        a = np.array(o)[None, :] * n + loc
        ok = np.ones(NLOC, bool)
        for e in range(DIM):
            ok &= (a[:, e] != 0) | (v[e] == 1)
            ok &= (a[:, e] != 2 * n - 1) | (v[e] == N - 1)
        mask.append(ok)
    return cells, np.concatenate(mask)


@pytest.mark.parametrize("prec", [SIPG_FP64, SIPG_FP32], ids=["fp64", "fp32"])
def test_apply_sampled_rows(solvers, blocks, prec):
    import torch
    s = solvers[prec]
    nd = s.ndofs()
    dt = torch.float64 if prec == SIPG_FP64 else torch.float32
    x = inputs.uniform(2000, nd)
    if prec == SIPG_FP32:
        x = x.astype(np.float32).astype(np.float64)
    y = torch.zeros(1, nd, dtype=dt, device="cuda")
    s.apply(NL - 1, dev(x, dt).view(1, -1), y)
    cells = sample_cells(2001)
    ref = block_apply(DIM, K, N, blocks, x, cells)
    got = host(y).reshape(-1, NLOC)[cells]
    if prec == SIPG_FP64:
        assert rel_inf(got, ref) < 1e-12
    else:
        absA = {key: (np.abs(v) if not isinstance(v, list) else [[np.abs(b) for b in r] for r in v])
                for key, v in blocks.items()}
        scale = block_apply(DIM, K, N, absA, np.abs(x), cells).max()
        assert np.abs(got - ref).max() < 64 * 6e-8 * scale


@pytest.mark.parametrize("colour", [0, 3, 5, 7])
@pytest.mark.parametrize("prec", [SIPG_FP64, SIPG_FP32], ids=["fp64", "fp32"])
def test_colour_pass_sampled_patches(solvers, blocks, prec, colour):
    import torch
    s = solvers[prec]
    nd = s.ndofs()
    dt = torch.float64 if prec == SIPG_FP64 else torch.float32
    b = inputs.normal(2010 + colour, nd)
    x0 = inputs.normal(2020 + colour, nd)
    if prec == SIPG_FP32:
        b = b.astype(np.float32).astype(np.float64)
        x0 = x0.astype(np.float32).astype(np.float64)
    xd = dev(x0, dt).view(1, -1)
    s.smooth_colour(NL - 1, colour, dev(b, dt).view(1, -1), xd)
    du = host(xd).ravel() - x0
    worst = 0.0
    for v in sample_patches(colour, 2030 + colour):
        cells, mask = patch_cells_and_mask(v)
        dofs = np.concatenate([np.arange(NLOC) + c * NLOC for c in cells])
        Ax = block_apply(DIM, K, N, blocks, x0, cells).ravel()
        r = b[dofs][mask] - Ax[mask]
        Aj = principal_block(DIM, K, N, blocks, cells)[np.ix_(mask, mask)]
        u = np.linalg.solve(Aj, r)
        got = du[dofs][mask]
        worst = max(worst, np.abs(got - u).max() / np.abs(u).max())
        # patch-boundary nodes of the patch cells are not touched by this patch
        # (and by no other patch of the colour)
        assert np.all(du[dofs][~mask] == 0.0)
    assert worst < (1e-10 if prec == SIPG_FP64 else 1e-4), worst


def test_vcycle_symmetric_fullsize(solvers):
    import torch
    s = solvers[SIPG_FP64]
    nd = s.ndofs()
    xa = dev(inputs.normal(2040, nd)).view(1, -1)
    xb = dev(inputs.normal(2041, nd)).view(1, -1)
    ba = torch.zeros_like(xa)
    bb = torch.zeros_like(xb)
    s.vcycle(xa, ba)
    s.vcycle(xb, bb)
    lhs = (ba * xb).sum().item()
    rhs = (xa * bb).sum().item()
    scale = (ba.norm() * xb.norm()).item()
    assert abs(lhs - rhs) < 1e-12 * scale


@pytest.fixture(scope="module")
def bench_problem():
    nd = (N * n) ** DIM
    X = node_coordinates(DIM, N, gauss_lobatto(K)[0])
    f = DIM * np.pi ** 2 * np.prod(np.sin(np.pi * X), axis=1) + inputs.uniform(2, nd)
    b = rhs_from_nodal(DIM, K, N, f)
    u = GlobalFD(DIM, K, N).solve(b)
    return b, u


@pytest.mark.parametrize("prec", [SIPG_FP64, SIPG_FP32], ids=["fp64", "mixed"])
def test_solve_fullsize_matches_direct(solvers, bench_problem, prec):
    import torch
    s = solvers[prec]
    b, u = bench_problem
    bd = dev(b).view(1, -1)
    x = torch.zeros_like(bd)
    # 1e-11 is close to the FP64 residual floor at this size (|A||x| / |b|
    # ~ 1e4 here); the solution is compared with the exact direct solve
    info = s.solve(bd, x, rtol=1e-11, maxit=60, allow_noconv=True)
    got = host(x).ravel()
    err = np.linalg.norm(got - u) / np.linalg.norm(u)
    print(f"prec={prec} rtol=1e-11: iterations={info.iterations} status={info.status} "
          f"rel_residual={info.rel_residual:.3e} err={err:.3e}")
    assert info.rel_residual <= 2e-11
    assert err < (1e-10 if prec == SIPG_FP64 else 1e-8), err
    # the benchmark's own stopping point (1e-10) is reported, with its error
    x.zero_()
    info = s.solve(bd, x, rtol=1e-10, maxit=100)
    err10 = np.linalg.norm(host(x).ravel() - u) / np.linalg.norm(u)
    print(f"prec={prec} iterations={info.iterations} nu={info.nu:.2f} err_at_1e-10={err10:.3e}")
    assert err10 < 1e-6
