"""Bind-time autotuning of the smoothing-step launch paths (sipg_tuning):
the recorded choices are valid, and a tuned handle solves to the same
solution as one with the default launch rules (SIPG_AUTOTUNE=0)."""
import numpy as np
import pytest

from gpu_helpers import dev, gpu_available, host, make

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

from paper_2405_18982_gb300 import SIPG_FP32, SIPG_FP64, inputs  # noqa: E402


@pytest.mark.parametrize("case", [(3, 3, 5, 5, SIPG_FP32), (3, 2, 4, 3, SIPG_FP64), (2, 4, 6, 5, SIPG_FP32)])
def test_choices_valid(case):
    dim, k, l2, nl, prec = case
    s = make(dim, k, l2, nl, prec=prec, graphs=1)
    assert s.tuning(0) == (-1, 0)  # the coarsest level is solved, not smoothed
    for lev in range(1, nl):
        path, tile = s.tuning(lev)
        assert path in (0, 1)
        assert tile in (0, 1, 2, 3, 4)
        if not (dim == 3 and prec == SIPG_FP32):
            assert tile == 0


@pytest.mark.parametrize("case", [(3, 3, 5, 5), (2, 3, 6, 5)])
def test_tuned_and_default_solve_agree(case, monkeypatch):
    import torch
    dim, k, l2, nl = case
    tuned = make(dim, k, l2, nl, prec=SIPG_FP32, graphs=1)
    monkeypatch.setenv("SIPG_AUTOTUNE", "0")
    plain = make(dim, k, l2, nl, prec=SIPG_FP32, graphs=1)
    monkeypatch.delenv("SIPG_AUTOTUNE")
    assert all(plain.tuning(lev) == (-1, 0) for lev in range(nl))
    b = dev(inputs.normal(1200, tuned.ndofs())).view(1, -1)
    xa, xb = torch.zeros_like(b), torch.zeros_like(b)
    ia = tuned.solve(b, xa, rtol=1e-10)
    ib = plain.solve(b, xb, rtol=1e-10)
    assert abs(ia.iterations - ib.iterations) <= 1
    ua, ub = host(xa).ravel(), host(xb).ravel()
    assert np.linalg.norm(ua - ub) <= 1e-8 * np.linalg.norm(ub)
