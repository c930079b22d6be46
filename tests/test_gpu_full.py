"""The paper's full-kernel (Sec. 3.1, Table 1) and clamped-kernel (Sec. 3.1,
Table 2 right) smoothers through the C ABI: FP32 colour passes and V-cycles
against the oracle, FCG and GMRES solves against the exact discrete
solution, and the fractional iteration counts of the tables' settings.
(FP64 colour passes: tests/test_gpu_parity.py; GMRES histories:
tests/test_gpu_gmres.py.)"""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from gpu_helpers import dev, gpu_available, host, make, rel_inf  # noqa: E402
from oracle.assembly import rhs_from_nodal  # noqa: E402
from oracle.direct import GlobalFD  # noqa: E402
from oracle.mg import Hierarchy, Level, fractional_iterations, gmres, smooth  # noqa: E402
from paper_2405_18982_gb300 import (SIPG_FP32, SIPG_FP64, SIPG_SMOOTHER_CLAMPED, SIPG_SMOOTHER_FULL,  # noqa: E402
                                    inputs)

KERNELS = {SIPG_SMOOTHER_FULL: "full", SIPG_SMOOTHER_CLAMPED: "clamped"}

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
CASES = [(2, 2, 4, 3), (2, 7, 3, 2), (3, 2, 3, 2), (3, 3, 3, 3), (3, 5, 2, 2)]
IDS = [f"d{d}k{k}N{1 << l}L{n}" for d, k, l, n in CASES]


@pytest.mark.parametrize("kernel", list(KERNELS), ids=list(KERNELS.values()))
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_full_colour_pass_fp32(case, kernel):
    import torch
    dim, k, l2, nl = case
    N = 1 << l2
    s = make(dim, k, l2, nl, prec=SIPG_FP32, smoother=kernel)
    lev = Level(dim, k, N, variant=KERNELS[kernel])
    b = inputs.normal(800, lev.ndof).astype(np.float32)
    x0 = inputs.normal(801, lev.ndof).astype(np.float32)
    bd = dev(b, torch.float32)
    xd = dev(x0, torch.float32)
    x = x0.astype(np.float64)
    for c in range(2 ** dim):
        s.smooth_colour(nl - 1, c, bd, xd)
        x = smooth(lev, x, b.astype(np.float64), colours=[c])
        assert np.abs(host(xd) - x).max() <= 1e-4 * np.abs(x - x0).max(), f"colour {c}"


@pytest.mark.parametrize("case", [(2, 5), (3, 5), (4, 4), (5, 4)], ids=lambda c: f"k{c[0]}N{1 << c[1]}")
def test_full_colour_pass_fp32_sampled(case):
    # the full kernel's 3D FP32 pass (register-direct all-rows kernels, one
    # launch for the interior and one for the boundary patches) on meshes
    # where a colour spans many CTAs: sampled patches (first and last of each
    # launch, every boundary type, random ones) against the oracle's dense
    # solve with the global residual, every DoF outside the colour's patch
    # cells bit-unchanged
    import torch
    from patch_sampling import PatchOracle, colour_touch_mask, sample_vertices
    k, l2 = case
    N = 1 << l2
    s = make(3, k, l2, l2, prec=SIPG_FP32, smoother=SIPG_SMOOTHER_FULL)
    nd = s.ndofs(l2 - 1)
    b = inputs.normal(810 + k, nd).astype(np.float32).astype(np.float64)
    x0 = inputs.normal(820 + k, nd).astype(np.float32).astype(np.float64)
    bd = dev(b, torch.float32).view(1, -1)
    po = PatchOracle(3, k, N, "full")
    for c in range(8):
        xd = dev(x0, torch.float32).view(1, -1)
        s.smooth_colour(l2 - 1, c, bd, xd)
        x1 = host(xd).ravel()
        touch = colour_touch_mask(3, k, N, c, full=True)
        assert np.array_equal(x1[~touch], x0[~touch]), f"colour {c} wrote outside its patch cells"
        du = x1 - x0
        for v in sample_vertices(3, N, c, 830 + c, 10):
            idx, u = po.update(v, b, x0)
            err = np.abs(du[idx] - u).max() / np.abs(u).max()
            assert err < 1e-4, (c, v, err)


@pytest.mark.parametrize("kernel", list(KERNELS), ids=list(KERNELS.values()))
@pytest.mark.parametrize("prec", [SIPG_FP64, SIPG_FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES[1:4], ids=IDS[1:4])
def test_full_vcycle(case, prec, kernel):
    import torch
    dim, k, l2, nl = case
    N = 1 << l2
    s = make(dim, k, l2, nl, prec=prec, smoother=kernel)
    H = Hierarchy(dim, k, N, nl, variant=KERNELS[kernel])
    dt = torch.float64 if prec == SIPG_FP64 else torch.float32
    b = inputs.normal(810, H.A.shape[0])
    if prec == SIPG_FP32:
        b = b.astype(np.float32).astype(np.float64)
    xd = dev(np.zeros_like(b), dt)
    s.vcycle(dev(b, dt), xd)
    assert rel_inf(host(xd), H.vcycle(b)) < (1e-10 if prec == SIPG_FP64 else 1e-4)


@pytest.mark.parametrize("kernel", list(KERNELS), ids=list(KERNELS.values()))
@pytest.mark.parametrize("prec", [SIPG_FP64, SIPG_FP32], ids=["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES[:4], ids=IDS[:4])
def test_full_kernel_solves(case, prec, kernel):
    dim, k, l2, nl = case
    if kernel == SIPG_SMOOTHER_CLAMPED and k < 3:
        pytest.skip("the clamped kernel's tables start at Q3; for Q2 its space is 2 functions per direction")
    N = 1 << l2
    s = make(dim, k, l2, nl, prec=prec, kappa=0.8, smoother=kernel)
    b = rhs_from_nodal(dim, k, N, inputs.normal(820, s.ndofs()))
    u = GlobalFD(dim, k, N, 0.8).solve(b)
    tol = 1e-10 if prec == SIPG_FP64 else 1e-8
    xd = dev(np.zeros_like(b))
    info = s.solve(dev(b), xd, rtol=1e-12, maxit=300)          # FCG: symmetric V-cycle
    assert info.status == 0 and rel_inf(host(xd), u) < tol
    xd = dev(np.zeros_like(b))
    info = s.gmres_solve(dev(b), xd, rtol=1e-12, maxit=300, restart=64)
    assert info.status == 0 and rel_inf(host(xd), u) < tol


def test_table1_setting_on_device():
    # Table 1 (full kernel): 3D, f = 1, GMRES to 1e-8.  At L = 3 the device
    # reproduces the oracle's nu; at L = 5 nu stays within a factor 1.6 of
    # the table and below the Dirichlet kernel's nu (Table 2's ordering).
    import torch
    ref = np.loadtxt(os.path.join(GOLDEN, "table1_full_nu.txt"))
    k, L = 3, 3
    N = 1 << L
    H = Hierarchy(3, k, N, L, variant="full")
    b = rhs_from_nodal(3, k, N, np.ones(H.A.shape[0]))
    _, h_ref = gmres(lambda v: H.A @ v, H.vcycle, b, rtol=1e-8, maxit=60)
    s = make(3, k, L, L, smoother=SIPG_SMOOTHER_FULL)
    info = s.gmres_solve(dev(b), dev(np.zeros_like(b)), rtol=1e-8, maxit=60)
    # nu comes from the last residual (1e-8 of the first), which carries the
    # rounding difference between the device's fast diagonalisation and the
    # oracle's Cholesky solves amplified by the residual reduction
    assert abs(info.nu - fractional_iterations(h_ref)) <= 1e-4 * fractional_iterations(h_ref)
    L = 5
    nus = {}
    for sm in (SIPG_SMOOTHER_FULL, 1):
        s = make(3, k, L, L, prec=SIPG_FP32, smoother=sm)
        f = torch.ones(1, s.ndofs(), dtype=torch.float64, device="cuda")
        bd = torch.zeros_like(f)
        s.rhs(f, bd)
        info = s.gmres_solve(bd, torch.zeros_like(f), rtol=1e-8, maxit=60)
        assert info.status == 0
        nus[sm] = info.nu
    printed = ref[L - 2, k - 2]
    assert printed / 1.6 <= nus[SIPG_SMOOTHER_FULL] <= printed * 1.6, (nus, printed)
    assert nus[SIPG_SMOOTHER_FULL] < nus[1]


def test_table2_clamped_setting_on_device():
    # Table 2, clamped kernel, with GMRES preconditioned from the left (the
    # reading under which the oracle reproduces the clamped column): at L = 3
    # the device reproduces the oracle's left-preconditioned history and nu;
    # at L = 5 (Q3 on 32^3 cells) nu is within 20 % of the printed 19.0,
    # not above the L = 3 value (the printed column falls from 22.7 to 19.0)
    # and above the Dirichlet kernel's.  The right-preconditioned device GMRES still
    # reproduces the oracle's right-preconditioned nu at L = 3.
    import torch
    ref = np.loadtxt(os.path.join(GOLDEN, "table2_clamped_nu.txt"))
    k, L = 3, 3
    N = 1 << L
    H = Hierarchy(3, k, N, L, variant="clamped")
    b = rhs_from_nodal(3, k, N, np.ones(H.A.shape[0]))
    s = make(3, k, L, L, smoother=SIPG_SMOOTHER_CLAMPED)
    nu3 = {}
    for left in (True, False):
        _, h_ref = gmres(lambda v: H.A @ v, H.vcycle, b, rtol=1e-8, maxit=100, restart=64,
                         side="left" if left else "right")
        nu3[left] = fractional_iterations(h_ref)
        info = s.gmres_solve(dev(b), dev(np.zeros_like(b)), rtol=1e-8, maxit=100, restart=64, left=left)
        assert info.status == 0 and info.iterations == len(h_ref) - 1
        # up to 42 GMRES steps: the last residual carries the rounding
        # difference of the local solves amplified by the residual reduction
        assert abs(info.nu - nu3[left]) <= 1e-3 * nu3[left], (left, info.nu, nu3[left])
        h = np.array(info.history[:len(h_ref)])
        assert np.allclose(h, h_ref, rtol=1e-5, atol=1e-12 * h_ref[0])
    L = 5
    nus = {}
    for sm in (SIPG_SMOOTHER_CLAMPED, 1):
        s = make(3, k, L, L, smoother=sm)
        f = torch.ones(1, s.ndofs(), dtype=torch.float64, device="cuda")
        bd = torch.zeros_like(f)
        s.rhs(f, bd)
        info = s.gmres_solve(bd, torch.zeros_like(f), rtol=1e-8, maxit=200, restart=64, left=True)
        assert info.status == 0
        nus[sm] = info.nu
    printed = ref[L - 2, k - 2]
    assert abs(nus[SIPG_SMOOTHER_CLAMPED] - printed) <= 0.2 * printed, (nus, printed)
    assert nus[SIPG_SMOOTHER_CLAMPED] <= nu3[True], (nus, nu3)
    assert nus[SIPG_SMOOTHER_CLAMPED] > nus[1]
