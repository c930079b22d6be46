"""sipg_dot_noalloc, the dot product for callers that cannot allocate device
memory (their allocator already owns it all, or a cudaMalloc would
synchronise the device on their latency path), checked through the C ABI
against sipg_dot, which uses the bound workspace as scratch.

This file is named to be collected last.  It must pass on its own in a fresh
process as well as after the other tests: the library's first call on the
device does the scratch address lookup, whichever test makes it.
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import dev, gpu_available, host, make

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


def _call(lib, name, *args):
    st = getattr(lib, name)(*args)
    assert st == 0, (name, st)


def test_noalloc_dot_matches_workspace_dot_twice():
    import torch
    from paper_2405_18982_gb300 import inputs, load
    lib = load()
    s = make(3, 2, 3, 2, nrhs=3)
    n = s.ndofs()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ref = torch.zeros(3, dtype=torch.float64, device="cuda")
    got = torch.zeros(3, dtype=torch.float64, device="cuda")
    for call in range(2):
        a = dev(inputs.normal_columns([990 + 3 * call, 991 + 3 * call, 992 + 3 * call], n))
        b = dev(inputs.normal_columns([995 + call, 996 + call, 997 + call], n))
        pa, pb = ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr())
        _call(lib, "sipg_dot", s.h, pa, pb, ctypes.c_void_p(ref.data_ptr()), stream)
        _call(lib, "sipg_dot_noalloc", s.h, pa, pb, ctypes.c_void_p(got.data_ptr()), stream)
        r, g = host(ref), host(got)
        exact = np.einsum("ij,ij->i", host(a), host(b))
        assert np.allclose(g, r, rtol=1e-13, atol=0), (call, g, r)
        assert np.allclose(g, exact, rtol=1e-12, atol=0)


def test_noalloc_dot_needs_no_workspace_and_rejects_oversize():
    import torch
    from paper_2405_18982_gb300 import _binding as B, inputs, load
    lib = load()
    # a handle that was created but never bound to a workspace
    p = B.sipg_params(2, 2, 3, 2, 1.0, 1.0, 0, 0, 2, 0)
    h = ctypes.c_void_p()
    assert lib.sipg_create(ctypes.byref(p), ctypes.byref(h)) == 0
    try:
        n = lib.sipg_ndofs(h, 1)
        a = dev(inputs.normal_columns([980, 981], n))
        out = torch.zeros(2, dtype=torch.float64, device="cuda")
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        st = lib.sipg_dot_noalloc(h, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(a.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), stream)
        assert st == 0
        assert np.allclose(host(out), np.sum(host(a) ** 2, axis=1), rtol=1e-12)
    finally:
        lib.sipg_destroy(h)
    big = B.sipg_params(2, 1, 2, 1, 1.0, 1.0, 0, 0, 65, 0)
    h = ctypes.c_void_p()
    assert lib.sipg_create(ctypes.byref(big), ctypes.byref(h)) == 0
    try:
        st = lib.sipg_dot_noalloc(h, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), None)
        assert st == B.SIPG_EINVAL
        assert b"64 columns" in lib.sipg_last_error(h)
    finally:
        lib.sipg_destroy(h)
