"""The C-ABI library builds, loads and exports every symbol include/cbp.h declares.

No GPU needed: only calls that fail argument validation before touching CUDA run here.
"""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2305_05286_gb300 import build, cbp

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "cbp.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cbp_[a-z_]+)\s*\(", src)))


def test_header_declares_the_binding_exports():
    assert declared_functions() == sorted(cbp.EXPORTS)


def test_library_exports_every_declared_symbol():
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for name in declared_functions():
        assert name in exported, name
    lib = C.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name)


def test_strerror_and_host_side_validation():
    L = cbp.lib()
    assert L.cbp_strerror(0) == b"success"
    assert L.cbp_strerror(-5) == b"workspace too small"
    h = C.c_void_p()
    base = np.array([[0, 0, -1], [-1, 0, 0]], np.int32)
    # invalid arguments are rejected before any CUDA call
    assert L.cbp_code_create(None, 2, 3, 4, C.byref(h)) == -1
    assert L.cbp_code_create(base.ctypes.data, 2, 3, 0, C.byref(h)) == -1
    bad = base.copy(); bad[0, 0] = 4
    assert L.cbp_code_create(bad.ctypes.data, 2, 3, 4, C.byref(h)) == -1         # shift >= Z
    deg1 = np.array([[0, -1, -1], [0, 0, 0]], np.int32)
    assert L.cbp_code_create(deg1.ctypes.data, 2, 3, 4, C.byref(h)) == -1        # degree-1 check
    empty = np.array([[0, 0, -1], [0, 0, -1]], np.int32)
    assert L.cbp_code_create(empty.ctypes.data, 2, 3, 4, C.byref(h)) == -1       # unused column
    big = np.zeros((2, 3), np.int32)
    assert L.cbp_code_create(big.ctypes.data, 2, 3, 2048, C.byref(h)) == -4      # Z > 1024
    assert h.value is None
    nb = C.c_size_t()
    assert L.cbp_workspace_bytes(None, 1, None, C.byref(nb)) == -1
    assert L.cbp_decode(None, None, None, None, 30, 1, None, 0, None) == -1
    assert L.cbp_phi(None, None, -1, None) == -1
    assert L.cbp_phi(None, None, 0, None) == 0
