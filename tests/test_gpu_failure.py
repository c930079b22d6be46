"""Failure detection without a GPU fault: bounded device waits report a
status the host reads, and the context stays usable afterwards."""
import numpy as np
import pytest

from gpu_helpers import dev, gpu_available, host, make, rel_inf

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


def test_bounded_barrier_times_out_and_context_survives():
    import ctypes
    import time
    import torch
    from oracle.assembly import rhs_from_nodal
    from oracle.direct import GlobalFD
    from paper_2405_18982_gb300 import _binding as B, inputs, load
    lib = load()
    s = make(3, 2, 3, 2)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.sipg_selftest_barrier(s.h, 0, stream) == B.SIPG_OK
    t0 = time.time()
    st = lib.sipg_selftest_barrier(s.h, 1, stream)   # a barrier nobody can open
    assert st == B.SIPG_ETIMEOUT
    assert time.time() - t0 < 30
    assert b"timed out" in lib.sipg_last_error(s.h)
    # the context and the handle still work
    f = inputs.normal(970, s.ndofs())
    b = rhs_from_nodal(3, 2, 8, f)
    x = dev(np.zeros_like(b))
    info = s.solve(dev(b), x, rtol=1e-10)
    assert info.status == 0
    assert rel_inf(host(x), GlobalFD(3, 2, 8).solve(b)) < 1e-8


def test_invalid_inputs_are_rejected_not_faulted():
    import ctypes
    import torch
    from paper_2405_18982_gb300 import _binding as B, load
    lib = load()
    s = make(2, 2, 3, 2)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.sipg_apply(s.h, 5, 0, ctypes.c_void_p(16), ctypes.c_void_p(32), stream) == B.SIPG_EINVAL
    assert lib.sipg_apply(s.h, 0, 7, ctypes.c_void_p(16), ctypes.c_void_p(32), stream) == B.SIPG_EINVAL
    assert lib.sipg_smooth_colour(s.h, 1, 0, 9, ctypes.c_void_p(16), ctypes.c_void_p(32), stream) == B.SIPG_EINVAL
    assert lib.sipg_restrict(s.h, 0, 0, ctypes.c_void_p(16), ctypes.c_void_p(32), stream) == B.SIPG_EINVAL
    assert lib.sipg_selftest_barrier(s.h, -1, stream) == B.SIPG_EINVAL
    x = torch.zeros(s.ndofs(), dtype=torch.float64, device="cuda")
    assert lib.sipg_solve(s.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), 1e-10, 10,
                          None, stream) == B.SIPG_EINVAL
