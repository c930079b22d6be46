"""GB300 (sm_103a) matrix-free multigrid for SIPG discontinuous Galerkin Poisson
problems on Cartesian meshes (after Cui & Kanschat, arXiv 2405.18982).

The compute path is the CUDA library ``_lib/libsipg.so`` (C ABI in
``include/sipg.h``).  This module is a thin binding: PyTorch supplies device
memory (the caller-owned workspace and vectors) and the current CUDA stream;
each method marshals pointers and calls the C entry point of the same name.
There is no CPU fallback: without the built library or a GPU every call
raises.
"""
import ctypes
from dataclasses import dataclass

from . import _binding as B
from ._binding import (SIPG_FP32, SIPG_FP64, SIPG_TF32, SIPG_SMOOTHER_CLAMPED, SIPG_SMOOTHER_CONSISTENT,
                       SIPG_SMOOTHER_FULL, SIPG_SMOOTHER_PAPER, SipgError, load)

__all__ = ["Params", "SIPG", "SIPGBatch", "SipgError", "SIPG_FP64", "SIPG_FP32", "SIPG_TF32",
           "SIPG_SMOOTHER_CONSISTENT", "SIPG_SMOOTHER_PAPER", "SIPG_SMOOTHER_FULL",
           "SIPG_SMOOTHER_CLAMPED", "load", "build"]


def build(force=False, verbose=False):
    """Compile libsipg.so for sm_103a (in-tree)."""
    from .build import build as _b
    return _b(force=force, verbose=verbose)


@dataclass
class Params:
    """Mirror of ``sipg_params`` (include/sipg.h)."""
    dim: int = 3
    degree: int = 3
    log2_cells: int = 3
    n_levels: int = 2
    kappa: float = 1.0
    penalty_factor: float = 1.0
    vcycle_precision: int = SIPG_FP64
    smoother: int = SIPG_SMOOTHER_CONSISTENT
    nrhs: int = 1
    use_graphs: int = 0

    def to_c(self):
        return B.sipg_params(self.dim, self.degree, self.log2_cells, self.n_levels, self.kappa,
                             self.penalty_factor, self.vcycle_precision, self.smoother, self.nrhs,
                             self.use_graphs)


@dataclass
class SolveInfo:
    iterations: int
    status: int
    rel_residual: float
    nu: float
    history: list


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _prec_of(t):
    import torch
    if t.dtype == torch.float64:
        return SIPG_FP64
    if t.dtype == torch.float32:
        return SIPG_FP32
    raise ValueError(f"unsupported dtype {t.dtype}")


class SIPG:
    """One SIPG multigrid problem (all levels) bound to caller-owned memory.

    ``SIPG(Params(...))`` creates the handle, allocates the workspace as a
    torch uint8 tensor on the current CUDA device and runs the device setup.
    """

    def __init__(self, params, device=None, stream=None):
        import torch
        self.lib = load()
        self._owned = True
        self.params = params
        self._cp = params.to_c()
        h = ctypes.c_void_p()
        st = self.lib.sipg_create(ctypes.byref(self._cp), ctypes.byref(h))
        if st != 0:
            raise SipgError(st, "sipg_create rejected the parameters")
        self.h = h
        self.device = torch.device(device) if device is not None else torch.device("cuda")
        nbytes = self.lib.sipg_workspace_bytes(self.h)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        self._ws_ptr = aligned
        self._check(self.lib.sipg_bind_workspace(self.h, ctypes.c_void_p(aligned), nbytes,
                                                 self._stream(stream)))

    # ------------------------------------------------------------ plumbing
    def _stream(self, stream):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        return ctypes.c_void_p(s.cuda_stream)

    def _check(self, st):
        if st != 0:
            msg = self.lib.sipg_last_error(self.h)
            raise SipgError(st, msg.decode() if msg else "")
        return st

    def close(self):
        if getattr(self, "h", None) and getattr(self, "_owned", False):
            self.lib.sipg_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ sizes
    def ndofs(self, level=None):
        if level is None:
            level = self.params.n_levels - 1
        return int(self.lib.sipg_ndofs(self.h, level))

    def launch_count(self):
        return int(self.lib.sipg_launch_count(self.h))

    def new_vector(self, level=None, dtype=None):
        import torch
        dtype = dtype or torch.float64
        return torch.zeros(self.params.nrhs, self.ndofs(level), dtype=dtype, device=self.device)

    # ------------------------------------------------------------ operators
    def rhs(self, f, b, stream=None):
        return self._check(self.lib.sipg_rhs(self.h, _ptr(f), _ptr(b), self._stream(stream)))

    def manufactured_source(self, f, stream=None):
        return self._check(self.lib.sipg_manufactured_source(self.h, _ptr(f), self._stream(stream)))

    def apply(self, level, x, y, stream=None):
        return self._check(self.lib.sipg_apply(self.h, level, _prec_of(x), _ptr(x), _ptr(y),
                                               self._stream(stream)))

    def residual(self, level, b, x, r, stream=None):
        return self._check(self.lib.sipg_residual(self.h, level, _prec_of(x), _ptr(b), _ptr(x), _ptr(r),
                                                  self._stream(stream)))

    def apply_penalty(self, x, y, stream=None):
        return self._check(self.lib.sipg_apply_penalty(self.h, _ptr(x), _ptr(y), self._stream(stream)))

    def smooth_colour(self, level, colour, b, x, stream=None):
        return self._check(self.lib.sipg_smooth_colour(self.h, level, _prec_of(x), colour, _ptr(b), _ptr(x),
                                                       self._stream(stream)))

    def smooth(self, level, b, x, reverse=False, stream=None):
        return self._check(self.lib.sipg_smooth(self.h, level, _prec_of(x), int(reverse), _ptr(b), _ptr(x),
                                                self._stream(stream)))

    def restrict(self, fine_level, rf, rc, stream=None):
        return self._check(self.lib.sipg_restrict(self.h, fine_level, _prec_of(rf), _ptr(rf), _ptr(rc),
                                                  self._stream(stream)))

    def prolongate_add(self, fine_level, ec, xf, stream=None):
        return self._check(self.lib.sipg_prolongate_add(self.h, fine_level, _prec_of(ec), _ptr(ec), _ptr(xf),
                                                        self._stream(stream)))

    def coarse_solve(self, b0, x0, stream=None):
        return self._check(self.lib.sipg_coarse_solve(self.h, _prec_of(b0), _ptr(b0), _ptr(x0),
                                                      self._stream(stream)))

    def vcycle(self, b, x, stream=None):
        return self._check(self.lib.sipg_vcycle(self.h, _prec_of(b), _ptr(b), _ptr(x), self._stream(stream)))

    def dot(self, a, b, out, stream=None):
        return self._check(self.lib.sipg_dot(self.h, _ptr(a), _ptr(b), _ptr(out), self._stream(stream)))

    # ------------------------------------------------------------ solvers
    def _solve(self, fn, b, x, rtol, maxit, stream, history, allow_noconv):
        hist = (ctypes.c_double * history)()
        info = B.sipg_info(0, 0, 0.0, 0.0, hist, history, 0)
        st = fn(self.h, _ptr(b), _ptr(x), rtol, maxit, ctypes.byref(info), self._stream(stream))
        if st != 0 and not (allow_noconv and st == B.SIPG_ENOCONV):
            self._check(st)
        return SolveInfo(info.iterations, info.status, info.rel_residual, info.nu,
                         [hist[i] for i in range(info.history_len)])

    def solve(self, b, x, rtol=1e-10, maxit=200, stream=None, history=256, allow_noconv=False, zero_start=False):
        """FCG to ||r|| <= rtol ||b||; x holds the initial guess, or with
        zero_start=True is output only (the iteration starts from x = 0 and
        skips the first residual apply: sipg_solve_zero)."""
        fn = self.lib.sipg_solve_zero if zero_start else self.lib.sipg_solve
        return self._solve(fn, b, x, rtol, maxit, stream, history, allow_noconv)

    def adjoint_solve(self, g, lam, rtol=1e-10, maxit=200, stream=None, history=256, allow_noconv=False):
        return self._solve(self.lib.sipg_adjoint_solve, g, lam, rtol, maxit, stream, history, allow_noconv)

    def gmres_workspace_bytes(self, restart=30):
        return int(self.lib.sipg_gmres_workspace_bytes(self.h, restart))

    def gmres_solve(self, b, x, rtol=1e-8, maxit=200, restart=30, stream=None, history=256,
                    allow_noconv=False, work=None, left=False):
        """GMRES preconditioned by the V-cycle (the paper's outer solver),
        from the right (sipg_gmres_solve) or with left=True from the left
        (sipg_gmres_solve_left); ``work`` (a CUDA uint8 tensor) is allocated
        here when not given or too small."""
        import torch
        nbytes = self.gmres_workspace_bytes(restart)
        if nbytes == 0:
            raise SipgError(B.SIPG_EINVAL, f"restart {restart} out of range")
        if work is None or work.numel() < nbytes + 256:
            work = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        aligned = (work.data_ptr() + 255) & ~255
        hist = (ctypes.c_double * history)()
        info = B.sipg_info(0, 0, 0.0, 0.0, hist, history, 0)
        fn = self.lib.sipg_gmres_solve_left if left else self.lib.sipg_gmres_solve
        st = fn(self.h, _ptr(b), _ptr(x), rtol, maxit, restart, ctypes.c_void_p(aligned), nbytes, ctypes.byref(info),
                self._stream(stream))
        if st != 0 and not (allow_noconv and st == B.SIPG_ENOCONV):
            self._check(st)
        return SolveInfo(info.iterations, info.status, info.rel_residual, info.nu,
                         [hist[i] for i in range(info.history_len)])

    def solve_host(self, f_host, u_host, rtol=1e-10, maxit=200, stream=None, history=256, allow_noconv=False):
        """f_host, u_host: CPU float64 tensors (pinned for async copies)."""
        if f_host.is_cuda or u_host.is_cuda:
            raise ValueError("solve_host takes host tensors")
        hist = (ctypes.c_double * history)()
        info = B.sipg_info(0, 0, 0.0, 0.0, hist, history, 0)
        st = self.lib.sipg_solve_host(self.h, ctypes.c_void_p(f_host.data_ptr()),
                                      ctypes.c_void_p(u_host.data_ptr()), rtol, maxit, ctypes.byref(info),
                                      self._stream(stream))
        if st != 0 and not (allow_noconv and st == B.SIPG_ENOCONV):
            self._check(st)
        return SolveInfo(info.iterations, info.status, info.rel_residual, info.nu,
                         [hist[i] for i in range(info.history_len)])

    def selftest_mma_tf32(self, a, b, d, stream=None):
        """Tensor-core self test (sipg_selftest_mma_tf32): d = a b^T for a
        (256, 16) and b (16, 16) float32 CUDA tensors, TF32 operands."""
        return self._check(self.lib.sipg_selftest_mma_tf32(self.h, _ptr(a), _ptr(b), _ptr(d), self._stream(stream)))

    def tuning(self, level, precision=None):
        """(path, tile) chosen by the bind-time autotuner for `level`."""
        prec = self.params.vcycle_precision if precision is None else precision
        path, tile = ctypes.c_int(0), ctypes.c_int(0)
        self._check(self.lib.sipg_tuning(self.h, level, prec, ctypes.byref(path), ctypes.byref(tile)))
        return path.value, tile.value

    def get_constants(self, level, which, ptype=0, cap=1 << 14, stream=None):
        import numpy as np
        buf = (ctypes.c_double * cap)()
        cnt = ctypes.c_int(0)
        self._check(self.lib.sipg_get_constants(self.h, level, which, ptype, buf, cap, ctypes.byref(cnt),
                                                self._stream(stream)))
        return np.array(buf[:min(cnt.value, cap)])


class SIPGBatch:
    """A ragged batch of independent problems (``sipg_batch_*``): one workspace
    for all members, solved together with ``solve`` (each member on its own
    stream, the flexible CG iterations advancing in lockstep)."""

    def __init__(self, params_list, device=None, stream=None):
        import torch
        self.lib = load()
        self.params = list(params_list)
        arr = (B.sipg_params * len(self.params))(*[p.to_c() for p in self.params])
        self._arr = arr
        h = ctypes.c_void_p()
        st = self.lib.sipg_batch_create(arr, len(self.params), ctypes.byref(h))
        if st != 0:
            raise SipgError(st, "sipg_batch_create rejected the parameters")
        self.h = h
        self.device = torch.device(device) if device is not None else torch.device("cuda")
        nbytes = self.lib.sipg_batch_workspace_bytes(self.h)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        aligned = (self.workspace.data_ptr() + 255) & ~255
        self._check(self.lib.sipg_batch_bind_workspace(self.h, ctypes.c_void_p(aligned), nbytes,
                                                       self._stream(stream)))
        self.members = []
        for i, p in enumerate(self.params):
            m = SIPG.__new__(SIPG)
            m.lib, m.params, m._owned, m.device = self.lib, p, False, self.device
            m.h = ctypes.c_void_p(self.lib.sipg_batch_member(self.h, i))
            self.members.append(m)

    def __len__(self):
        return len(self.members)

    def _stream(self, stream):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        return ctypes.c_void_p(s.cuda_stream)

    def _check(self, st):
        if st != 0:
            msg = self.lib.sipg_batch_last_error(self.h)
            raise SipgError(st, msg.decode() if msg else "")
        return st

    def solve(self, bs, xs, rtol=1e-10, maxit=200, stream=None, history=64, allow_noconv=False):
        """bs, xs: lists of member vectors (contiguous CUDA float64)."""
        n = len(self.members)
        if len(bs) != n or len(xs) != n:
            raise ValueError("one b and one x per member")
        bp = (ctypes.c_void_p * n)(*[_ptr(b).value for b in bs])
        xp = (ctypes.c_void_p * n)(*[_ptr(x).value for x in xs])
        hists = [(ctypes.c_double * history)() for _ in range(n)]
        infos = (B.sipg_info * n)(*[B.sipg_info(0, 0, 0.0, 0.0, hists[i], history, 0) for i in range(n)])
        st = self.lib.sipg_batch_solve(self.h, bp, xp, rtol, maxit, infos, self._stream(stream))
        if st != 0 and not (allow_noconv and st == B.SIPG_ENOCONV):
            self._check(st)
        return [SolveInfo(infos[i].iterations, infos[i].status, infos[i].rel_residual, infos[i].nu,
                          [hists[i][j] for j in range(infos[i].history_len)]) for i in range(n)]

    def close(self):
        for m in getattr(self, "members", []):
            m.h = None
        if getattr(self, "h", None):
            self.lib.sipg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
