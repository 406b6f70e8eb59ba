"""The C-ABI library loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def _declared():
    names = []
    for h in HEADERS:
        txt = open(h).read()
        names += re.findall(r"BFX_API\s+[\w\s\*]+?\b(bfx_\w+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def so():
    from paper_1904_06376_b300 import build as b

    path = b.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for must in ("bfx_split", "bfx_gemm_bf16xN", "bfx_gemm_presplit", "bfx_sgemm_simt"):
        assert must in names


def test_every_declared_symbol_exported(so):
    missing = [n for n in _declared() if not hasattr(so, n)]
    assert not missing, missing


def test_only_api_symbols_exported(so):
    """Internal symbols stay hidden (built with -fvisibility=hidden)."""
    import subprocess

    from paper_1904_06376_b300 import build as b

    out = subprocess.run(["nm", "-D", "--defined-only", b.LIB], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    bfx_syms = {s for s in exported if s.startswith("bfx_")}
    assert bfx_syms == set(_declared())


def test_host_only_calls(so):
    so.bfx_version.restype = ctypes.c_int
    assert so.bfx_version() >= 100
    so.bfx_status_string.restype = ctypes.c_char_p
    so.bfx_status_string.argtypes = [ctypes.c_int]
    assert so.bfx_status_string(0) == b"ok"
    assert so.bfx_status_string(99) == b"unknown status"
    ws = so.bfx_gemm_workspace_size
    ws.restype = ctypes.c_size_t
    ws.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
    # x6: 3 planes each of A (m x kp) and B^T (n x kp), kp = k rounded up to 8, 256-byte planes
    assert ws(6, 128, 256, 64) == 3 * (128 * 64 + 256 * 64) * 2
    assert ws(3, 1, 1, 1) == 2 * (128 + 128) * 2
    assert ws(0, 10, 10, 10) == 0  # FP32 SIMT needs no workspace
    assert ws(7, 10, 10, 10) == 0  # invalid mode


def test_invalid_arguments_rejected_before_any_launch(so):
    """Argument errors are reported synchronously without touching a GPU."""
    f = so.bfx_split
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    assert f(-1, 4, None, 4, 3, None, None, None, 4, None) == 1
    assert f(4, 4, None, 4, 4, None, None, None, 4, None) == 1
    assert f(4, 4, None, 4, 3, None, None, None, 4, None) == 1  # null pointers
    assert f(0, 4, None, 4, 3, None, None, None, 4, None) == 0  # empty: nothing to do
    g = so.bfx_gemm_bf16xN
    g.restype = ctypes.c_int
    assert g(5, 4, 4, 4, ctypes.c_float(1.0), None, ctypes.c_int64(4), None, ctypes.c_int64(4),
             ctypes.c_float(0.0), None, ctypes.c_int64(4), None, ctypes.c_size_t(0), None) == 1
