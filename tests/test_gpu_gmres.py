"""GMRES, the paper's outer solver (Sec. 3.3, Tables 1 and 2), through the C
ABI: step-by-step residual histories against the oracle's GMRES (same
V-cycle, both local-residual variants), solutions against the exact discrete
solution, restarts, argument errors, and the fractional iteration count of
the paper's Dirichlet-kernel setting against Table 2."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from gpu_helpers import dev, gpu_available, host, make, rel_inf  # noqa: E402
from oracle.assembly import rhs_from_nodal  # noqa: E402
from oracle.direct import GlobalFD  # noqa: E402
from oracle.mg import Hierarchy, fractional_iterations, gmres  # noqa: E402
from paper_2405_18982_gb300 import SIPG_FP32, SIPG_FP64, inputs  # noqa: E402

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
# (dim, k, log2 N, levels)
CASES = [(2, 2, 4, 3), (2, 4, 3, 2), (3, 2, 3, 2), (3, 3, 3, 3)]
IDS = [f"d{d}k{k}N{1 << l}L{n}" for d, k, l, n in CASES]
_HIER = {}


def hierarchy(dim, k, N, nl, kappa=1.0, variant="consistent"):
    key = (dim, k, N, nl, kappa, variant)
    if key not in _HIER:
        _HIER[key] = Hierarchy(dim, k, N, nl, kappa=kappa, variant=variant)
    return _HIER[key]


@pytest.mark.parametrize("graphs", [0, 1], ids=["host-steps", "device-cycles"])
@pytest.mark.parametrize("variant", [0, 1, 2], ids=["consistent", "paper", "full"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_gmres_history_matches_oracle(case, variant, graphs):
    # same V-cycle (FP64), same GMRES: the residual after every step agrees
    # with the oracle's (the device orthogonalises by classical Gram-Schmidt
    # applied twice, the oracle by modified Gram-Schmidt: equal in exact
    # arithmetic); with graphs every restart cycle runs on the device
    dim, k, l2, nl = case
    N = 1 << l2
    s = make(dim, k, l2, nl, kappa=1.1, smoother=variant, graphs=graphs)
    H = hierarchy(dim, k, N, nl, kappa=1.1, variant=("consistent", "paper", "full")[variant])
    b = rhs_from_nodal(dim, k, N, inputs.normal(700, H.A.shape[0]))
    x_ref, h_ref = gmres(lambda v: H.A @ v, H.vcycle, b, rtol=1e-10, maxit=100, restart=30)
    xd = dev(np.zeros_like(b))
    info = s.gmres_solve(dev(b), xd, rtol=1e-10, maxit=100, restart=30)
    assert info.status == 0 and info.rel_residual <= 1e-10
    assert info.iterations == len(h_ref) - 1
    h = np.array(info.history)
    assert len(h) == len(h_ref)
    assert np.all(np.abs(h - h_ref) <= 1e-6 * np.asarray(h_ref) + 1e-13 * h_ref[0])
    assert rel_inf(host(xd), x_ref) < 1e-7
    assert abs(info.nu - fractional_iterations(h_ref)) <= 1e-4 * fractional_iterations(h_ref)


@pytest.mark.parametrize("prec,variant", [(SIPG_FP64, 0), (SIPG_FP64, 1), (SIPG_FP32, 0), (SIPG_FP32, 1)],
                         ids=["fp64-consistent", "fp64-paper", "mixed-consistent", "mixed-paper"])
@pytest.mark.parametrize("case", CASES[::2], ids=IDS[::2])
def test_gmres_solution_matches_exact(case, prec, variant):
    dim, k, l2, nl = case
    N = 1 << l2
    s = make(dim, k, l2, nl, prec=prec, kappa=0.8, smoother=variant)
    b = rhs_from_nodal(dim, k, N, inputs.normal(720, s.ndofs()))
    xd = dev(np.zeros_like(b))
    info = s.gmres_solve(dev(b), xd, rtol=1e-12, maxit=200, restart=40)
    assert info.status == 0 and info.rel_residual <= 1e-12
    u = GlobalFD(dim, k, N, 0.8).solve(b)
    assert rel_inf(host(xd), u) < (1e-10 if prec == SIPG_FP64 else 1e-8)


@pytest.mark.parametrize("graphs", [0, 1], ids=["host-steps", "device-cycles"])
def test_gmres_restarts_and_warm_start(graphs):
    dim, k, l2, nl = 3, 3, 3, 2
    N = 1 << l2
    s = make(dim, k, l2, nl, smoother=1, graphs=graphs)
    b = rhs_from_nodal(dim, k, N, inputs.normal(730, s.ndofs()))
    u = GlobalFD(dim, k, N).solve(b)
    xd = dev(np.zeros_like(b))
    info = s.gmres_solve(dev(b), xd, rtol=1e-11, maxit=200, restart=2)
    assert info.status == 0 and info.iterations > 2
    h = np.array(info.history)
    assert np.all(h[1:] <= h[:-1] * (1 + 1e-12))
    assert rel_inf(host(xd), u) < 1e-9
    # warm start from the solution: converged before the first step
    info2 = s.gmres_solve(dev(b), xd, rtol=1e-10, maxit=10, restart=5)
    assert info2.iterations == 0 and info2.rel_residual <= 1e-10


@pytest.mark.parametrize("prec,left", [(SIPG_FP64, False), (SIPG_FP32, False), (SIPG_FP64, True)],
                         ids=["fp64-right", "mixed-right", "fp64-left"])
def test_device_cycles_equal_host_steps(prec, left, monkeypatch):
    # the same GMRES driven step by step from the host and as one graph
    # launch per restart cycle: same steps, histories and solutions up to
    # rounding (the rotations run on the host in one and on the device in
    # the other); short restarts and a step limit that ends inside a cycle.
    # Both handles take the default launch paths (no autotuning), so that
    # their FP32 V-cycles run the same kernels and round alike.
    monkeypatch.setenv("SIPG_AUTOTUNE", "0")
    dim, k, l2, nl = 3, 3, 4, 3
    N = 1 << l2
    b = rhs_from_nodal(dim, k, N, inputs.normal(760, (N * (k + 1)) ** 3))
    runs = {}
    for graphs in (0, 1):
        s = make(dim, k, l2, nl, prec=prec, smoother=0, graphs=graphs)
        xd = dev(np.zeros_like(b))
        info = s.gmres_solve(dev(b), xd, rtol=1e-11, maxit=100, restart=4, left=left)
        x2 = dev(np.zeros_like(b))
        info2 = s.gmres_solve(dev(b), x2, rtol=1e-11, maxit=7, restart=3, left=left, allow_noconv=True)
        # a second solve reuses the recorded cycle graph
        x3 = dev(np.zeros_like(b))
        info3 = s.gmres_solve(dev(b), x3, rtol=1e-11, maxit=100, restart=4, left=left)
        runs[graphs] = (info, host(xd), info2, host(x2), info3, host(x3))
    (i0, x0, j0, y0, _, _), (i1, x1, j1, y1, k1, z1) = runs[0], runs[1]
    assert i0.status == 0 and i1.status == 0 and i1.iterations == i0.iterations > 4
    h0, h1 = np.array(i0.history), np.array(i1.history)
    assert len(h0) == len(h1) and np.all(np.abs(h1 - h0) <= 1e-9 * h0 + 1e-14 * h0[0])
    assert rel_inf(x1, x0) < 1e-10
    assert j0.status == j1.status and j1.iterations == j0.iterations == 7
    assert np.allclose(j1.history, j0.history, rtol=1e-9, atol=1e-14 * h0[0])
    assert rel_inf(y1, y0) < 1e-10
    assert k1.iterations == i1.iterations and np.array_equal(z1, x1)
    u = GlobalFD(dim, k, N).solve(b)
    assert rel_inf(x1, u) < (1e-9 if prec == SIPG_FP64 else 1e-8)


def test_gmres_errors():
    import ctypes

    import torch
    from paper_2405_18982_gb300 import SipgError, _binding as B
    s = make(2, 2, 3, 2)
    n = s.ndofs()
    b = dev(inputs.normal(740, n))
    x = dev(np.zeros(n))
    info = s.gmres_solve(b, x, rtol=1e-14, maxit=1, allow_noconv=True)
    assert info.status == B.SIPG_ENOCONV and info.iterations == 1
    assert s.gmres_workspace_bytes(0) == 0 and s.gmres_workspace_bytes(65) == 0
    need = s.gmres_workspace_bytes(4)
    assert need >= 9 * n * 8
    work = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    base = (work.data_ptr() + 255) & ~255
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = (s.h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), 1e-8, 100, 4)
    assert s.lib.sipg_gmres_solve(*args, ctypes.c_void_p(base), need - 8, None, stream) == B.SIPG_EINVAL
    assert s.lib.sipg_gmres_solve(*args, ctypes.c_void_p(base + 16), need, None, stream) == B.SIPG_EINVAL
    assert s.lib.sipg_gmres_solve(*args, ctypes.c_void_p(base), need, None, stream) == 0
    multi = make(2, 2, 3, 2, nrhs=2)
    with pytest.raises(SipgError):
        multi.gmres_solve(dev(np.zeros(2 * n)), dev(np.zeros(2 * n)))
    # a non-finite right-hand side ends in a clean status, and the handle
    # stays usable
    bad = inputs.normal(741, n)
    bad[5] = np.nan
    x.zero_()
    with pytest.raises(SipgError) as err:
        s.gmres_solve(dev(bad), x, rtol=1e-8, maxit=10)
    assert err.value.status == B.SIPG_EBREAKDOWN
    x.zero_()
    assert s.gmres_solve(b, x, rtol=1e-8, maxit=100).status == 0


@pytest.mark.parametrize("prec", [SIPG_FP64, SIPG_FP32], ids=["fp64", "mixed"])
def test_table2_setting_on_device(prec):
    # Table 2's Dirichlet column: 3D, f = 1, GMRES to 1e-8 preconditioned by
    # the V-cycle with the paper's Dirichlet-kernel residual.  At L = 3 the
    # device reproduces the oracle's nu (itself within 20 % of the table);
    # at L = 5, beyond the oracle's reach, nu stays within 20 % of the table.
    import torch
    ref = np.loadtxt(os.path.join(GOLDEN, "table2_dirichlet_nu.txt"))
    k, L = 3, 3
    N = 1 << L
    H = hierarchy(3, k, N, L, variant="paper")
    b = rhs_from_nodal(3, k, N, np.ones(H.A.shape[0]))
    _, h_ref = gmres(lambda v: H.A @ v, H.vcycle, b, rtol=1e-8, maxit=60)
    s = make(3, k, L, L, prec=prec, smoother=1)
    info = s.gmres_solve(dev(b), dev(np.zeros_like(b)), rtol=1e-8, maxit=60)
    # nu comes from the last residual (1e-8 of the first), which carries the
    # rounding difference between the device's fast diagonalisation and the
    # oracle's Cholesky solves amplified by the residual reduction
    tol = 1e-4 if prec == SIPG_FP64 else 2e-2
    assert abs(info.nu - fractional_iterations(h_ref)) <= tol * fractional_iterations(h_ref)
    L = 5
    s = make(3, k, L, L, prec=prec, smoother=1)
    f = torch.ones(1, s.ndofs(), dtype=torch.float64, device="cuda")
    bd = torch.zeros_like(f)
    s.rhs(f, bd)
    info = s.gmres_solve(bd, torch.zeros_like(f), rtol=1e-8, maxit=60)
    printed = ref[L - 2, k - 2]
    assert info.status == 0 and abs(info.nu - printed) <= 0.2 * printed, (info.nu, printed)
    # Table 4's single-GPU column prints 5.8 for this setting
    ref4 = np.loadtxt(os.path.join(GOLDEN, "table4_local_nu.txt"))
    assert abs(info.nu - ref4[L - 2, 1]) <= 0.1 * ref4[L - 2, 1], info.nu
