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
    good = sipg_params(3, 3, 6, 6, 1.0, 1.0, 1, 0, 1, 0)
    assert lib.sipg_create(ctypes.byref(good), ctypes.byref(h)) == 0 and h.value
    assert lib.sipg_ndofs(h, 5) == 64 ** 3 * 64
    assert lib.sipg_ndofs(h, 0) == 2 ** 3 * 64
    ws = lib.sipg_workspace_bytes(h)
    assert ws > 6 * 64 ** 3 * 64 * 8
    # calls before binding a workspace are rejected, not crashed
    assert lib.sipg_apply(h, 0, 0, ctypes.c_void_p(16), ctypes.c_void_p(32), None) == -8
    assert b"workspace" in lib.sipg_last_error(h)
    lib.sipg_destroy(h)
    assert lib.sipg_version().startswith(b"sipg")
