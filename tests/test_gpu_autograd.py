"""Gradients of J = 1/2 ||u - u_obs||^2 through the differentiable solve
(hand-written adjoint backward) against the FP64 oracle gradient (exact
global fast-diagonalisation solves) and FP64 central differences."""
import numpy as np
import pytest

from gpu_helpers import dev, gpu_available, host

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

from oracle.adjoint import loss_and_gradients  # noqa: E402
from oracle.assembly import penalty  # noqa: E402
from paper_2405_18982_gb300 import SIPG_FP32, SIPG_FP64, inputs  # noqa: E402


def _problem(dim, k, l2, nl, prec, seed):
    import torch
    from paper_2405_18982_gb300.autograd import SolverCache
    cache = SolverCache(dim, k, l2, nl, vcycle_precision=prec)
    N = 1 << l2
    nd = N ** dim * (k + 1) ** dim
    f = inputs.normal(seed, nd)
    u_obs = inputs.normal(seed + 1, nd) * 1e-2
    kappa = inputs.scalar_uniform(seed + 2, 0.5, 2.0)
    gamma = penalty(k, N, 1.0)
    return cache, f, u_obs, kappa, gamma


@pytest.mark.parametrize("case", [(2, 3, 3, 2), (3, 2, 3, 2), (3, 3, 2, 2)])
@pytest.mark.parametrize("prec", [SIPG_FP64, SIPG_FP32], ids=["fp64", "mixed"])
def test_gradients_match_oracle(case, prec):
    import torch
    from paper_2405_18982_gb300.autograd import sipg_solve
    dim, k, l2, nl = case
    cache, f, u_obs, kappa, gamma = _problem(dim, k, l2, nl, prec, 1000)
    ft = dev(f).view(1, -1).requires_grad_(True)
    kt = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
    gt = torch.tensor(gamma, dtype=torch.float64, requires_grad=True)
    u = sipg_solve(ft, kt, gt, cache, rtol=1e-13)
    J = 0.5 * ((u - dev(u_obs).view(1, -1)) ** 2).sum()
    J.backward()
    J_ref, gf_ref, gk_ref, gg_ref, u_ref, _ = loss_and_gradients(dim, k, 1 << l2, f, kappa, gamma, u_obs)
    assert abs(J.item() - J_ref) < 1e-9 * abs(J_ref)
    assert np.abs(host(ft.grad).ravel() - gf_ref).max() < 1e-8 * np.abs(gf_ref).max()
    assert abs(kt.grad.item() - gk_ref) < 1e-8 * abs(gk_ref)
    assert abs(gt.grad.item() - gg_ref) < 1e-7 * abs(gg_ref)


def test_gradients_match_central_differences():
    import torch
    from paper_2405_18982_gb300.autograd import sipg_solve
    dim, k, l2, nl = 3, 3, 3, 2
    cache, f, u_obs, kappa, gamma = _problem(dim, k, l2, nl, SIPG_FP64, 1010)
    uo = dev(u_obs).view(1, -1)

    def J(ff, kk, gg):
        with torch.no_grad():
            u = sipg_solve(ff, kk, gg, cache, rtol=1e-13)
            return 0.5 * ((u - uo) ** 2).sum().item()

    ft = dev(f).view(1, -1).requires_grad_(True)
    kt = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
    gt = torch.tensor(gamma, dtype=torch.float64, requires_grad=True)
    u = sipg_solve(ft, kt, gt, cache, rtol=1e-13)
    (0.5 * ((u - uo) ** 2).sum()).backward()
    step = 1e-6
    fd_k = (J(ft.detach(), kappa * (1 + step), gamma) - J(ft.detach(), kappa * (1 - step), gamma)) / (2 * kappa * step)
    fd_g = (J(ft.detach(), kappa, gamma * (1 + step)) - J(ft.detach(), kappa, gamma * (1 - step))) / (2 * gamma * step)
    d = dev(inputs.normal(1020, ft.shape[1])).view(1, -1)
    fd_f = (J(ft.detach() + step * d, kappa, gamma) - J(ft.detach() - step * d, kappa, gamma)) / (2 * step)
    assert abs(fd_k - kt.grad.item()) < 1e-5 * abs(kt.grad.item())
    assert abs(fd_g - gt.grad.item()) < 1e-5 * abs(gt.grad.item())
    assert abs(fd_f - (ft.grad * d).sum().item()) < 1e-5 * abs((ft.grad * d).sum().item())


def test_fp32_source_gets_fp32_gradient():
    import torch
    from paper_2405_18982_gb300.autograd import sipg_solve
    cache, f, u_obs, kappa, gamma = _problem(2, 2, 4, 3, SIPG_FP32, 1030)
    ft = dev(f, torch.float32).view(1, -1).requires_grad_(True)
    u = sipg_solve(ft, kappa, gamma, cache, rtol=1e-10)
    assert u.dtype == torch.float64
    (0.5 * ((u - dev(u_obs).view(1, -1)) ** 2).sum()).backward()
    assert ft.grad.dtype == torch.float32 and torch.isfinite(ft.grad).all()


def test_c5_fullsize_gradients():
    # 3D Q3 on 32^3 cells (2.1M DoFs), 5 levels, mixed precision: u_obs from a
    # solve with f_obs ~ N(0,1) (seed 5, kappa = 1); f ~ N(0,1) (seed 6) as an
    # FP32 tensor, kappa ~ U[0.5, 2] (seed 7), gamma = 2k(k+1)/h.  Gradients
    # against the oracle's exact ones and FP64 central differences (step 1e-6)
    import torch
    from oracle.adjoint import forward, loss_and_gradients_blocks
    from paper_2405_18982_gb300.autograd import SolverCache, sipg_solve
    dim, k, l2, nl = 3, 3, 5, 5
    N = 1 << l2
    nd = N ** dim * (k + 1) ** dim
    gamma = penalty(k, N, 1.0)
    u_obs = forward(dim, k, N, inputs.normal(5, nd), 1.0, gamma)[0]
    f = inputs.normal(6, nd).astype(np.float32)
    kappa = inputs.scalar_uniform(7, 0.5, 2.0)
    cache = SolverCache(dim, k, l2, nl, vcycle_precision=SIPG_FP32)
    uo = dev(u_obs).view(1, -1)
    ft = dev(f, torch.float32).view(1, -1).requires_grad_(True)
    kt = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
    gt = torch.tensor(gamma, dtype=torch.float64, requires_grad=True)
    u = sipg_solve(ft, kt, gt, cache, rtol=1e-11)
    J = 0.5 * ((u - uo) ** 2).sum()
    J.backward()
    J_ref, gf_ref, gk_ref, gg_ref, _, _ = loss_and_gradients_blocks(dim, k, N, f.astype(np.float64), kappa, gamma,
                                                                     u_obs)
    print(f"C5: J={J.item():.6e} ref={J_ref:.6e} dJ/dkappa={kt.grad.item():.6e} ref={gk_ref:.6e} "
          f"dJ/dgamma={gt.grad.item():.6e} ref={gg_ref:.6e}")
    assert abs(J.item() - J_ref) < 1e-8 * abs(J_ref)
    assert ft.grad.dtype == torch.float32
    assert np.abs(host(ft.grad).ravel() - gf_ref).max() < 1e-5 * np.abs(gf_ref).max()
    assert abs(kt.grad.item() - gk_ref) < 1e-7 * abs(gk_ref)
    assert abs(gt.grad.item() - gg_ref) < 1e-6 * abs(gg_ref)

    def Jval(kk, gg):
        with torch.no_grad():
            uu = sipg_solve(ft.detach(), kk, gg, cache, rtol=1e-11)
            return 0.5 * ((uu - uo) ** 2).sum().item()

    step = 1e-6
    fd_k = (Jval(kappa * (1 + step), gamma) - Jval(kappa * (1 - step), gamma)) / (2 * kappa * step)
    fd_g = (Jval(kappa, gamma * (1 + step)) - Jval(kappa, gamma * (1 - step))) / (2 * gamma * step)
    assert abs(fd_k - kt.grad.item()) < 1e-4 * abs(kt.grad.item())
    assert abs(fd_g - gt.grad.item()) < 1e-4 * abs(gt.grad.item())
