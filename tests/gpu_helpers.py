"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np

try:
    import torch
except Exception:  # pragma: no cover
    torch = None


def gpu_available():
    return torch is not None and torch.cuda.is_available()


def make(dim, k, log2N, nlev, prec=0, kappa=1.0, eta=1.0, nrhs=1, smoother=0, graphs=0):
    from paper_2405_18982_gb300 import SIPG, Params
    return SIPG(Params(dim=dim, degree=k, log2_cells=log2N, n_levels=nlev, kappa=kappa,
                       penalty_factor=eta, vcycle_precision=prec, smoother=smoother, nrhs=nrhs,
                       use_graphs=graphs))


def dev(a, dtype=None):
    dtype = dtype or torch.float64
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().double().cpu().numpy()


def rel_inf(a, b):
    """max |a - b| / max |b|"""
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))
