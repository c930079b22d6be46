"""The C-ABI library loads (without a GPU) and exports every entry point that
include/sipg.h declares; the ctypes binding declares exactly those."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sipg.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(sipg_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2405_18982_gb300 import build
    path = build()
    return ctypes.CDLL(path)


def test_header_parses():
    names = declared_functions()
    assert "sipg_create" in names and "sipg_solve" in names and len(names) >= 20


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_matches_header():
    from paper_2405_18982_gb300._binding import SIGNATURES
    assert sorted(SIGNATURES) == declared_functions()


def test_host_only_calls_without_gpu(lib):
    # parameter validation and sizing need no GPU
    from paper_2405_18982_gb300._binding import SIGNATURES, sipg_params
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = res, args
    h = ctypes.c_void_p()
    bad = sipg_params(4, 3, 3, 2, 1.0, 1.0, 0, 0, 1, 0)
    assert lib.sipg_create(ctypes.byref(bad), ctypes.byref(h)) == -1 and not h.value
    bad = sipg_params(3, 3, 3, 4, 1.0, 1.0, 0, 0, 1, 0)   # coarsest level 1 cell
    assert lib.sipg_create(ctypes.byref(bad), ctypes.byref(h)) == -1
    bad = sipg_params(3, 3, 3, 2, -1.0, 1.0, 0, 0, 1, 0)  # kappa <= 0
    assert lib.sipg_create(ctypes.byref(bad), ctypes.byref(h)) == -1
    bad = sipg_params(2, 1, 3, 2, 1.0, 1.0, 0, 3, 1, 0)   # clamped kernel with k = 1: empty space
    assert lib.sipg_create(ctypes.byref(bad), ctypes.byref(h)) == -1
    bad = sipg_params(2, 2, 3, 2, 1.0, 1.0, 0, 4, 1, 0)   # no smoother 4
    assert lib.sipg_create(ctypes.byref(bad), ctypes.byref(h)) == -1
    ok = sipg_params(2, 2, 3, 2, 1.0, 1.0, 0, 3, 1, 0)
    assert lib.sipg_create(ctypes.byref(ok), ctypes.byref(h)) == 0
    lib.sipg_destroy(h)
    good = sipg_params(3, 3, 6, 6, 1.0, 1.0, 1, 0, 1, 0)
    assert lib.sipg_create(ctypes.byref(good), ctypes.byref(h)) == 0 and h.value
    assert lib.sipg_ndofs(h, 5) == 64 ** 3 * 64
    assert lib.sipg_ndofs(h, 0) == 2 ** 3 * 64
    ws = lib.sipg_workspace_bytes(h)
    assert ws > 6 * 64 ** 3 * 64 * 8
    # calls before binding a workspace are rejected, not crashed
    assert lib.sipg_apply(h, 0, 0, ctypes.c_void_p(16), ctypes.c_void_p(32), None) == -8
    assert b"workspace" in lib.sipg_last_error(h)
    # GMRES: restart bounds, workspace >= 2 restart + 1 finest-level vectors,
    # and no solve before binding
    nf = 64 ** 3 * 64
    assert lib.sipg_gmres_workspace_bytes(h, 0) == 0 and lib.sipg_gmres_workspace_bytes(h, 65) == 0
    assert lib.sipg_gmres_workspace_bytes(h, 1) >= 3 * nf * 8
    assert lib.sipg_gmres_workspace_bytes(h, 64) >= 129 * nf * 8
    assert lib.sipg_gmres_solve(h, ctypes.c_void_p(16), ctypes.c_void_p(32), 1e-8, 10, 4,
                                ctypes.c_void_p(256), 1 << 40, None, None) == -8
    lib.sipg_destroy(h)
    assert lib.sipg_version().startswith(b"sipg")


def test_batch_host_only_calls_without_gpu(lib):
    from paper_2405_18982_gb300._binding import SIGNATURES, sipg_params
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = res, args
    b = ctypes.c_void_p()
    arr = (sipg_params * 3)(sipg_params(2, 2, 5, 5, 1.0, 1.0, 1, 0, 1, 1),
                            sipg_params(2, 6, 9, 9, 1.0, 1.0, 1, 0, 1, 1),
                            sipg_params(2, 4, 7, 7, 1.0, 1.0, 1, 0, 1, 1))
    assert lib.sipg_batch_create(arr, 0, ctypes.byref(b)) == -1 and not b.value
    bad = (sipg_params * 2)(arr[0], sipg_params(2, 9, 5, 5, 1.0, 1.0, 1, 0, 1, 1))  # degree 9
    assert lib.sipg_batch_create(bad, 2, ctypes.byref(b)) == -1 and not b.value
    assert lib.sipg_batch_create(arr, 3, ctypes.byref(b)) == 0 and b.value
    assert lib.sipg_batch_count(b) == 3
    total = 0
    for i, (L, k) in enumerate([(5, 2), (9, 6), (7, 4)]):
        m = lib.sipg_batch_member(b, i)
        assert m and lib.sipg_ndofs(m, L - 1) == (1 << L) ** 2 * (k + 1) ** 2
        total += (lib.sipg_workspace_bytes(m) + 255) // 256 * 256
    assert not lib.sipg_batch_member(b, 3)
    # (the fused path is opt-in: by default the members' workspaces only)
    assert lib.sipg_batch_workspace_bytes(b) == total
    # solving before binding is rejected
    ptrs = (ctypes.c_void_p * 3)(16, 16, 16)
    xs = (ctypes.c_void_p * 3)(32, 32, 32)
    assert lib.sipg_batch_solve(b, ptrs, xs, 1e-10, 10, None, None) == -8
    assert b"bound" in lib.sipg_batch_last_error(b)
    lib.sipg_batch_destroy(b)


def test_tuning_query_without_gpu(lib):
    from paper_2405_18982_gb300._binding import SIGNATURES, sipg_params
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = res, args
    h = ctypes.c_void_p()
    assert lib.sipg_create(ctypes.byref(sipg_params(3, 3, 4, 3, 1.0, 1.0, 1, 0, 1, 0)), ctypes.byref(h)) == 0
    path, tile = ctypes.c_int(7), ctypes.c_int(7)
    # not bound, so not tuned: default rules
    assert lib.sipg_tuning(h, 2, 1, ctypes.byref(path), ctypes.byref(tile)) == 0
    assert (path.value, tile.value) == (-1, 0)
    assert lib.sipg_tuning(h, 3, 1, ctypes.byref(path), ctypes.byref(tile)) == -1  # no level 3
    assert lib.sipg_tuning(h, 0, 5, ctypes.byref(path), ctypes.byref(tile)) == -1  # bad precision
    lib.sipg_destroy(h)


def test_smoother_choices_and_gmres_sizes_without_gpu(lib):
    from paper_2405_18982_gb300._binding import SIGNATURES, sipg_params
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = res, args
    h = ctypes.c_void_p()
    for dim in (2, 3):
        for k in range(1, 8):
            for sm in range(4):
                p = sipg_params(dim, k, 3, 3, 1.0, 1.0, 0, sm, 1, 0)   # coarsest level 2 cells
                st = lib.sipg_create(ctypes.byref(p), ctypes.byref(h))
                if sm == 3 and k < 2:
                    assert st == -1 and not h.value
                    continue
                assert st == 0, (dim, k, sm)
                nf = lib.sipg_ndofs(h, 2)
                sizes = [lib.sipg_gmres_workspace_bytes(h, m) for m in (1, 2, 30, 64)]
                assert all(a < b for a, b in zip(sizes, sizes[1:]))
                for m, size in zip((1, 2, 30, 64), sizes):
                    assert size >= (2 * m + 1) * nf * 8
                lib.sipg_destroy(h)
