"""ctypes front end of the CPU oracle (gfe_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline leg use it; the product library never imports it.  It shares no
code with the CUDA path.

Result convention (arXiv 1806.04211, Eq. (echelon)): for A in GF(p)^{m x n}
    rank r, rho (pivot rows, ascending), ups (pivot columns, ascending),
    M (r x r), K ((m-r) x r), R (r x (n-r)), optional dense E (m x n), T (m x m)
with T = (M 0; K 1) P_rho and T A = E = (-RREF(A); 0).
GF(2) inputs and outputs are bit-packed int64 words (bit c%64 of word c/64).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gfe_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lib = None

_i64 = ctypes.c_int64
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile gfe_oracle.c into liborc.so next to it (plain gcc -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_echelon_u8.argtypes = [ctypes.c_int, _i64, _i64, _p, _i64, _p, _p, _p,
                                     _p, _i64, _p, _i64, _p, _i64, _p, _i64, _p, _i64]
        L.orc_echelon_gf2.argtypes = [_i64, _i64, _p, _i64, _p, _p, _p,
                                      _p, _i64, _p, _i64, _p, _i64, _p, _i64, _p, _i64]
        L.orc_certify_u8.argtypes = [ctypes.c_int, _i64, _i64, _p, _i64, _i64, _p, _p,
                                     _p, _i64, _p, _i64, _p, _i64, ctypes.c_int, ctypes.c_uint64]
        L.orc_certify_gf2.argtypes = [_i64, _i64, _p, _i64, _i64, _p, _p,
                                      _p, _i64, _p, _i64, _p, _i64, ctypes.c_uint64]
        for f in (L.orc_echelon_u8, L.orc_echelon_gf2, L.orc_certify_u8, L.orc_certify_gf2):
            f.restype = ctypes.c_int
        L.orc_is_prime.argtypes = [ctypes.c_int]
        L.orc_is_prime.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def echelon(A: np.ndarray, p: int, want_E: bool = False, want_T: bool = False) -> dict:
    """Echelon form with transformation of a uint8 matrix over GF(p), p > 2 or 2."""
    A = np.ascontiguousarray(A, dtype=np.uint8)
    m, n = A.shape
    rm = min(m, n)
    rank = np.zeros(1, np.int64)
    prow = np.zeros(max(rm, 1), np.int64)
    pcol = np.zeros(max(rm, 1), np.int64)
    M = np.zeros((max(rm, 1), max(rm, 1)), np.uint8)
    K = np.zeros((max(m, 1), max(rm, 1)), np.uint8)
    R = np.zeros((max(rm, 1), max(n, 1)), np.uint8)
    E = np.zeros((m, n), np.uint8) if want_E else None
    T = np.zeros((m, m), np.uint8) if want_T else None
    rc = lib().orc_echelon_u8(p, m, n, _ptr(A), n, rank.ctypes.data, prow.ctypes.data,
                              pcol.ctypes.data, M.ctypes.data, M.shape[1], K.ctypes.data,
                              K.shape[1], R.ctypes.data, R.shape[1], _ptr(E), n, _ptr(T), m)
    if rc:
        raise ValueError("oracle rejected the input (p=%d, %dx%d)" % (p, m, n))
    r = int(rank[0])
    out = dict(rank=r, rho=prow[:r].copy(), ups=pcol[:r].copy(), M=M[:r, :r].copy(),
               K=K[:m - r, :r].copy(), R=R[:r, :n - r].copy())
    if want_E:
        out["E"] = E
    if want_T:
        out["T"] = T
    return out


def _wpr(n: int) -> int:
    w = (n + 63) // 64
    return w + (w & 1)


def echelon_gf2(Aw: np.ndarray, m: int, n: int, want_E: bool = False, want_T: bool = False) -> dict:
    """Bit-packed GF(2) version; Aw is m x ldw int64/uint64 words."""
    Aw = np.ascontiguousarray(Aw).view(np.uint64)
    assert Aw.shape[0] == m and Aw.shape[1] * 64 >= n
    rm = min(m, n)
    rank = np.zeros(1, np.int64)
    prow = np.zeros(max(rm, 1), np.int64)
    pcol = np.zeros(max(rm, 1), np.int64)
    wr, wn, wm = _wpr(rm), _wpr(n), _wpr(m)
    M = np.zeros((max(rm, 1), wr), np.uint64)
    K = np.zeros((max(m, 1), wr), np.uint64)
    R = np.zeros((max(rm, 1), wn), np.uint64)
    E = np.zeros((m, wn), np.uint64) if want_E else None
    T = np.zeros((m, wm), np.uint64) if want_T else None
    rc = lib().orc_echelon_gf2(m, n, Aw.ctypes.data, Aw.shape[1], rank.ctypes.data,
                               prow.ctypes.data, pcol.ctypes.data, M.ctypes.data, wr,
                               K.ctypes.data, wr, R.ctypes.data, wn, _ptr(E), wn, _ptr(T), wm)
    if rc:
        raise ValueError("oracle rejected the input")
    r = int(rank[0])
    out = dict(rank=r, rho=prow[:r].copy(), ups=pcol[:r].copy(),
               M=M[:r, :_wpr(r)].copy(), K=K[:m - r, :_wpr(r)].copy(),
               R=R[:r, :_wpr(n - r)].copy())
    if want_E:
        out["E"] = E
    if want_T:
        out["T"] = T
    return out


def certify(A: np.ndarray, p: int, res: dict, nvec: int = 16, seed: int = 1) -> int:
    """Certificate check of a claimed result for a uint8 A; 0 = pass."""
    A = np.ascontiguousarray(A, dtype=np.uint8)
    m, n = A.shape
    r = int(res["rank"])
    rho = np.ascontiguousarray(res["rho"], dtype=np.int64)
    ups = np.ascontiguousarray(res["ups"], dtype=np.int64)
    M = np.ascontiguousarray(res["M"], dtype=np.uint8).reshape(r, r)
    K = np.ascontiguousarray(res["K"], dtype=np.uint8).reshape(m - r, r)
    R = np.ascontiguousarray(res["R"], dtype=np.uint8).reshape(r, n - r)
    return lib().orc_certify_u8(p, m, n, A.ctypes.data, n, r, rho.ctypes.data, ups.ctypes.data,
                                M.ctypes.data, max(r, 1), K.ctypes.data, max(r, 1),
                                R.ctypes.data, max(n - r, 1), nvec, seed)


def certify_gf2(Aw: np.ndarray, m: int, n: int, res: dict, seed: int = 1) -> int:
    """Certificate check of a claimed bit-packed GF(2) result; 0 = pass."""
    Aw = np.ascontiguousarray(Aw).view(np.uint64)
    r = int(res["rank"])
    rho = np.ascontiguousarray(res["rho"], dtype=np.int64)
    ups = np.ascontiguousarray(res["ups"], dtype=np.int64)
    M = np.ascontiguousarray(res["M"]).view(np.uint64)
    K = np.ascontiguousarray(res["K"]).view(np.uint64)
    R = np.ascontiguousarray(res["R"]).view(np.uint64)
    return lib().orc_certify_gf2(m, n, Aw.ctypes.data, Aw.shape[1], r, rho.ctypes.data,
                                 ups.ctypes.data, M.ctypes.data, M.shape[1] if M.ndim == 2 else 1,
                                 K.ctypes.data, K.shape[1] if K.ndim == 2 else 1,
                                 R.ctypes.data, R.shape[1] if R.ndim == 2 else 1, seed)


# --------------------------------------------------------------------------
# helpers for tests: bit (un)packing with numpy
# --------------------------------------------------------------------------

def unpack_bits(W: np.ndarray, ncols: int) -> np.ndarray:
    W = np.ascontiguousarray(W).view(np.uint64)
    if W.ndim == 1:
        W = W.reshape(1, -1)
    b = np.unpackbits(W.view(np.uint8).reshape(W.shape[0], -1), axis=1, bitorder="little")
    return b[:, :ncols].astype(np.uint8)


def pack_bits(B: np.ndarray, ldw: int | None = None) -> np.ndarray:
    B = np.asarray(B, dtype=np.uint8)
    m, n = B.shape
    if ldw is None:
        ldw = _wpr(n)
    pad = np.zeros((m, ldw * 64), np.uint8)
    pad[:, :n] = B
    return np.packbits(pad, axis=1, bitorder="little").view(np.uint64).reshape(m, ldw)
