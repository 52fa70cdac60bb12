"""ctypes front end of the CPU oracle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use this
module.  It compiles ``cbp_oracle.cpp`` with the host C++ compiler (no fused
multiply-add contraction, no fast-math) into ``oracle/_build/liboracle.so`` and
exposes the decoders on numpy arrays.  It imports nothing from the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cbp_oracle.cpp")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")

ALGS = {"cbp_sp": 0, "cbp_nms": 1, "lbp_nms": 2, "fbp_sp": 3, "lbp_sp": 4, "cbp_sp_omega": 5}
STOPS = {"syndrome": 0, "none": 1, "window": 2}
COUNTERS = ("sweeps", "b2v", "v2c", "c2b", "sums", "products", "c2v", "flush")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle library if it is missing or older than its source."""
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-pthread", "-o", tmp, SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            i32p, u8p, i64p = (np.ctypeslib.ndpointer(dtype=t, flags="C_CONTIGUOUS")
                               for t in (np.int32, np.uint8, np.int64))
            f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
            f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
            L.orc_code_create.restype = P
            L.orc_code_create.argtypes = [i32p, C.c_int, C.c_int, C.c_int]
            L.orc_code_destroy.argtypes = [P]
            L.orc_code_dims.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
            L.orc_code_edges.argtypes = [P, i32p, i32p]
            L.orc_decode_f32.restype = C.c_int
            L.orc_decode_f32.argtypes = [P, C.c_int, f32p, C.c_int, C.c_int, C.c_int, C.c_float,
                                         u8p, i32p, P, P, P, C.c_int]
            L.orc_decode_f64.restype = C.c_int
            L.orc_decode_f64.argtypes = [P, C.c_int, f64p, C.c_int, C.c_int, C.c_int, C.c_double,
                                         u8p, i32p, P, P, P, C.c_int]
            L.orc_cbp_trace_f64.restype = C.c_int
            L.orc_cbp_trace_f64.argtypes = [P, f64p, C.c_int, f64p, u8p, f64p, f64p]
            L.orc_weighted_f64.restype = C.c_int
            L.orc_weighted_f64.argtypes = [P, f64p, f64p, C.c_int, C.c_int, f64p]
            L.orc_weighted_f32.restype = C.c_int
            L.orc_weighted_f32.argtypes = [P, f32p, f32p, C.c_int, C.c_int, f32p]
            L.orc_weighted_grad_f64.restype = C.c_int
            L.orc_weighted_grad_f64.argtypes = [P, f64p, f64p, C.c_int, C.c_int, f64p, f64p, f64p]
            L.orc_phi_f32.argtypes = [f32p, f32p, C.c_int64]
            L.orc_phi_f64.argtypes = [f64p, f64p, C.c_int64]
            L.orc_phi_table_f32.restype = C.c_int
            L.orc_phi_table_f32.argtypes = [P, C.c_int]
            L.orc_phi_xlo_f32.restype = C.c_float
            L.orc_phi_xlo_f64.restype = C.c_double
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class OracleCode:
    """Expanded Tanner graph of a QC base matrix, held by the oracle library."""

    def __init__(self, base, Z: int):
        base = np.ascontiguousarray(np.asarray(base, dtype=np.int32))
        self._lib = lib()
        self._h = self._lib.orc_code_create(base, base.shape[0], base.shape[1], int(Z))
        if not self._h:
            raise ValueError("oracle rejected the base matrix")
        n, m, e = C.c_int(), C.c_int(), C.c_int()
        self._lib.orc_code_dims(self._h, C.byref(n), C.byref(m), C.byref(e))
        self.N, self.M, self.E = n.value, m.value, e.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_code_destroy(h)
            self._h = None

    def edges(self):
        echk = np.zeros(self.E, np.int32)
        evar = np.zeros(self.E, np.int32)
        self._lib.orc_code_edges(self._h, echk, evar)
        return echk, evar

    def decode(self, llr, alg="cbp_sp", max_iter=30, stop="syndrome", alpha=0.75,
               precision=32, soft=True, threads=1):
        """Decode frames ``llr`` [F, N].  Returns a dict of numpy arrays:
        hard uint8 [F, N], iters int32 [F], soft [F, N], flags uint8 [F], counts."""
        dt = np.float32 if precision == 32 else np.float64
        llr = np.ascontiguousarray(np.asarray(llr, dtype=dt).reshape(-1, self.N))
        F = llr.shape[0]
        hard = np.zeros((F, self.N), np.uint8)
        iters = np.zeros(F, np.int32)
        sft = np.zeros((F, self.N), dt) if soft else None
        flags = np.zeros(F, np.uint8)
        counts = np.zeros(len(COUNTERS), np.int64)
        fn = self._lib.orc_decode_f32 if precision == 32 else self._lib.orc_decode_f64
        rc = fn(self._h, ALGS[alg], llr, F, int(max_iter), STOPS[stop], alpha, hard, iters,
                _ptr(sft), _ptr(flags), _ptr(counts), int(threads))
        if rc != 0:
            raise ValueError(f"oracle decode failed ({rc})")
        return {"hard": hard, "iters": iters, "soft": sft, "flags": flags,
                "counts": dict(zip(COUNTERS, counts.tolist()))}

    def weighted(self, llr, w, T: int, precision: int = 64):
        """Weighted CBP, T sweeps: flushed posterior [F, N].  w: [T, mb] scales."""
        dt = np.float64 if precision == 64 else np.float32
        llr = np.ascontiguousarray(np.asarray(llr, dtype=dt).reshape(-1, self.N))
        w = np.ascontiguousarray(np.asarray(w, dtype=dt).reshape(-1))
        out = np.zeros_like(llr)
        fn = self._lib.orc_weighted_f64 if precision == 64 else self._lib.orc_weighted_f32
        if fn(self._h, llr, w, int(T), llr.shape[0], out) != 0:
            raise ValueError("weighted forward failed")
        return out

    def weighted_grad(self, llr, w, T: int, grad_soft):
        """FP64 adjoint: (grad_w [T, mb] summed over frames, grad_llr [F, N])."""
        llr = np.ascontiguousarray(np.asarray(llr, dtype=np.float64).reshape(-1, self.N))
        w = np.ascontiguousarray(np.asarray(w, dtype=np.float64).reshape(-1))
        gs = np.ascontiguousarray(np.asarray(grad_soft, dtype=np.float64).reshape(llr.shape))
        gw = np.zeros_like(w)
        gl = np.zeros_like(llr)
        if self._lib.orc_weighted_grad_f64(self._h, llr, w, int(T), llr.shape[0], gs, gw, gl) != 0:
            raise ValueError("weighted adjoint failed")
        return gw.reshape(int(T), -1), gl

    def trace(self, llr, sweeps: int):
        """FP64 CBP on one frame for exactly ``sweeps`` sweeps: (S, sigma, Q per edge, R per edge)."""
        llr = np.ascontiguousarray(np.asarray(llr, dtype=np.float64).reshape(self.N))
        S = np.zeros(self.M)
        sig = np.zeros(self.M, np.uint8)
        q = np.zeros(self.E)
        r = np.zeros(self.E)
        if self._lib.orc_cbp_trace_f64(self._h, llr, int(sweeps), S, sig, q, r) != 0:
            raise ValueError("trace failed")
        return S, sig, q, r


def phi32(x) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    y = np.empty_like(x)
    lib().orc_phi_f32(x.reshape(-1), y.reshape(-1), x.size)
    return y


def phi64(x) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    y = np.empty_like(x)
    lib().orc_phi_f64(x.reshape(-1), y.reshape(-1), x.size)
    return y


def phi_table() -> np.ndarray:
    n = lib().orc_phi_table_f32(None, 0)
    t = np.zeros(n, np.float32)
    lib().orc_phi_table_f32(t.ctypes.data_as(C.c_void_p), n)
    return t.reshape(-1, 4)


def xlo32() -> float:
    return float(lib().orc_phi_xlo_f32())
