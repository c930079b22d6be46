"""Tensor-core (TF32) path of the 3D colour pass (SIPG_TF32).

1. The MMA building block: one CTA computes D = A B^T (A 256 x 16, B 16 x 16,
   TF32 operands, FP32 accumulation) through the operand layouts, MMA issue,
   mbarrier completion and tensor-memory loads that the colour pass uses.
   TF32 products are exact in FP32, so D must equal the FP64 product of the
   TF32-rounded operands to the FP32 rounding of a 16-term sum.
2. Colour passes of the 3D Dirichlet kernel with the TF32 local solve (Q7;
   other degrees keep the FP32 kernel, so a TF32 handle solves them too),
   element by element against the oracle's dense patch solves (sampled
   patches, every DoF outside the colour's spaces unchanged), and different
   from the FP32 kernel's result (the tensor-core kernel ran).
3. Mixed solves with the TF32 V-cycle reach 1e-10 in the FP64 outer CG and
   match the exact solution to 1e-8.

Tolerance of 2: each of the six eigenvector sweeps rounds its operands to
TF32 (unit u = 2^-11) and sums p = 14 products in FP32, so a sweep's output
carries a relative error of about 2u in the norm of its input; six sweeps,
the eigenvalue scaling and the growth by the (M-orthonormal, not
orthogonal) eigenvector matrices give about 12u |S||S^T| ~ 1e-2 in the worst
element relative to the largest; we ask 1e-2 of the max-norm relative error
of each sampled patch's correction."""
import numpy as np
import pytest

from gpu_helpers import dev, gpu_available, host, make

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

from oracle.assembly import rhs_from_nodal  # noqa: E402
from oracle.direct import GlobalFD  # noqa: E402
from paper_2405_18982_gb300 import SIPG_FP32, SIPG_TF32, inputs  # noqa: E402
from patch_sampling import PatchOracle, colour_touch_mask, sample_vertices  # noqa: E402

TOL_TF32 = 1e-2


def tf32(a):
    """Round FP32 values to TF32 (10 stored mantissa bits), to nearest with
    ties away from zero: add half of the last kept bit to the magnitude and
    truncate."""
    bits = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    return ((bits + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


def test_mma_selftest_matches_fp64_product():
    import torch
    s = make(3, 7, 1, 1, prec=SIPG_TF32)
    A = inputs.normal(5000, 256 * 16).astype(np.float32).reshape(256, 16)
    B = inputs.normal(5001, 16 * 16).astype(np.float32).reshape(16, 16)
    A[3, :] *= 1e3                      # rows and columns of very different scale
    B[:, 5] *= 1e-3
    d = torch.zeros(256, 16, dtype=torch.float32, device="cuda")
    s.selftest_mma_tf32(dev(A, torch.float32), dev(B, torch.float32), d)
    got = host(d)
    At, Bt = tf32(A).astype(np.float64), tf32(B).astype(np.float64)
    ref = At @ Bt.T
    scale = np.abs(At) @ np.abs(Bt).T
    assert np.all(np.abs(got - ref) <= 16 * 2.0 ** -24 * scale + 1e-30), np.abs(got - ref).max()
    # TF32 and not FP32 operands: the rounding is visible in the product
    assert np.abs(got - A.astype(np.float64) @ B.astype(np.float64).T).max() > 0


@pytest.mark.parametrize("k", [7])
@pytest.mark.parametrize("variant", ["consistent", "paper"])
def test_tf32_colour_pass(variant, k):
    import torch
    from paper_2405_18982_gb300 import SIPG_SMOOTHER_CONSISTENT, SIPG_SMOOTHER_PAPER
    dim, l2 = 3, 4
    N = 1 << l2
    sm = SIPG_SMOOTHER_CONSISTENT if variant == "consistent" else SIPG_SMOOTHER_PAPER
    s = make(dim, k, l2, l2, prec=SIPG_TF32, smoother=sm)
    s32 = make(dim, k, l2, l2, prec=SIPG_FP32, smoother=sm)
    nd = s.ndofs(l2 - 1)
    b = inputs.normal(5010, nd).astype(np.float32).astype(np.float64)
    x0 = inputs.normal(5011, nd).astype(np.float32).astype(np.float64)
    bd = dev(b, torch.float32).view(1, -1)
    po = PatchOracle(dim, k, N, variant)
    worst = 0.0
    for c in range(8):
        xd = dev(x0, torch.float32).view(1, -1)
        s.smooth_colour(l2 - 1, c, bd, xd)
        x1 = host(xd).ravel()
        xe = dev(x0, torch.float32).view(1, -1)
        s32.smooth_colour(l2 - 1, c, bd, xe)
        x32 = host(xe).ravel()
        touch = colour_touch_mask(dim, k, N, c)
        assert np.array_equal(x1[~touch], x0[~touch])
        if c == 0:      # colour 0 has interior patches only: all of them on the tensor cores
            assert np.abs(x1 - x32).max() > 0
        du = x1 - x0
        for v in sample_vertices(dim, N, c, 5020 + c, 10 if k == 7 else 16):
            idx, u = po.update(v, b, x0)
            err = np.abs(du[idx] - u).max() / np.abs(u).max()
            worst = max(worst, err)
            assert err < TOL_TF32, (c, v, err)
    print(f"TF32 colour passes, Q{k} {N}^3 {variant}: worst sampled-patch error {worst:.2e}")


@pytest.mark.parametrize("case", [(3, 7, 3, 3), (3, 7, 4, 4), (3, 5, 4, 4)], ids=["q7n8", "q7n16", "q5n16"])
def test_tf32_mixed_solve_matches_exact(case):
    dim, k, l2, nl = case
    N = 1 << l2
    s = make(dim, k, l2, nl, prec=SIPG_TF32)
    f = inputs.normal(5030, s.ndofs())
    b = rhs_from_nodal(dim, k, N, f)
    xd = dev(np.zeros_like(b))
    info = s.solve(dev(b), xd, rtol=1e-12, maxit=100)
    u = GlobalFD(dim, k, N).solve(b)
    err = np.abs(host(xd) - u).max() / np.abs(u).max()
    assert info.rel_residual <= 1e-12 and err < 1e-8, (info, err)
