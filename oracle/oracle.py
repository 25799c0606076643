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
_SRC_OMP = os.path.join(_HERE, "gfe_oracle_omp.c")
_LIB_OMP = os.path.join(_HERE, "liborc_omp.so")
_lib = None
_lib_omp = None

_i64 = ctypes.c_int64
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile gfe_oracle.c into liborc.so next to it (plain gcc -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def build_omp(force: bool = False) -> str:
    """Compile gfe_oracle_omp.c (the oracle's GF(2) algorithm on all host
    cores, a timing baseline) into liborc_omp.so (gcc -O2 -fopenmp)."""
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < os.path.getmtime(_SRC_OMP):
        tmp = _LIB_OMP + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", _SRC_OMP, "-o", tmp])
        os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


def lib_omp():
    global _lib_omp
    if _lib_omp is None:
        build_omp()
        L = ctypes.CDLL(_LIB_OMP)
        L.orc_echelon_gf2_omp.argtypes = [_i64, _i64, _p, _i64, _p, _p, _p, _p, _i64, _p, _i64, _p, _i64]
        L.orc_echelon_gf2_omp.restype = ctypes.c_int
        L.orc_omp_threads.argtypes = []
        L.orc_omp_threads.restype = ctypes.c_int
        _lib_omp = L
    return _lib_omp


def omp_threads() -> int:
    """Threads the OpenMP baseline runs on (OMP_NUM_THREADS, else all cores)."""
    return int(lib_omp().orc_omp_threads())


def echelon_gf2_omp(Aw: np.ndarray, m: int, n: int) -> dict:
    """The bit-packed GF(2) oracle algorithm on all host cores (OpenMP):
    a timing baseline with the same outputs as echelon_gf2 (no E, T)."""
    Aw = np.ascontiguousarray(Aw).view(np.uint64)
    assert Aw.shape[0] == m and Aw.shape[1] * 64 >= n
    rm = min(m, n)
    rank = np.zeros(1, np.int64)
    prow = np.zeros(max(rm, 1), np.int64)
    pcol = np.zeros(max(rm, 1), np.int64)
    wr, wn = _wpr(rm), _wpr(n)
    M = np.zeros((max(rm, 1), wr), np.uint64)
    K = np.zeros((max(m, 1), wr), np.uint64)
    R = np.zeros((max(rm, 1), wn), np.uint64)
    rc = lib_omp().orc_echelon_gf2_omp(m, n, Aw.ctypes.data, Aw.shape[1], rank.ctypes.data, prow.ctypes.data,
                                       pcol.ctypes.data, M.ctypes.data, wr, K.ctypes.data, wr, R.ctypes.data, wn)
    if rc:
        raise ValueError("oracle rejected the input")
    r = int(rank[0])
    return dict(rank=r, rho=prow[:r].copy(), ups=pcol[:r].copy(), M=M[:r, :_wpr(r)].copy(),
                K=K[:m - r, :_wpr(r)].copy(), R=R[:r, :_wpr(n - r)].copy())


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


# --------------------------------------------------------------------------
# solving and kernels from the echelon result (the paper's variant list,
# Section 1: the transformation matrix gives the null space and solutions)
# --------------------------------------------------------------------------

def _complement(idx: np.ndarray, n: int) -> np.ndarray:
    mask = np.ones(n, dtype=bool)
    mask[np.asarray(idx, dtype=np.int64)] = False
    return np.nonzero(mask)[0]


def nullspace_left(A: np.ndarray, p: int) -> np.ndarray:
    """Basis of {y : y A = 0} as the rows of (K 1) P_rho, i.e. rows r..m-1 of
    T in Eq. (echelon) (Section 3.1): T A = E and those rows of E are zero.
    Row t has K[t, s] at column rho_s and 1 at column rho_bar_t, so the basis
    is the unique one that is the identity on the columns rho_bar."""
    A = np.ascontiguousarray(A, dtype=np.uint8)
    m = A.shape[0]
    res = echelon(A, p)
    r, rho = res["rank"], res["rho"]
    nbar = _complement(rho, m)
    N = np.zeros((m - r, m), np.uint8)
    if m - r:
        N[:, rho] = res["K"]
        N[np.arange(m - r), nbar] = 1
    return N


def nullspace_right(A: np.ndarray, p: int) -> np.ndarray:
    """Basis of {x : A x = 0}, one basis vector per row ((n-r) x n).  Since
    T is invertible, A x = 0 iff E_top x = 0, and row l of E_top = -RREF(A)
    reads -x[Ups_l] + sum_j R[l, j] x[Ups_bar_j] = 0.  Basis vector j is 1 at
    the non-pivot column Ups_bar_j, 0 at the other non-pivot columns and
    R[l, j] at the pivot column Ups_l: the unique basis that is the identity
    on the columns Ups_bar."""
    A = np.ascontiguousarray(A, dtype=np.uint8)
    n = A.shape[1]
    res = echelon(A, p)
    r, ups = res["rank"], res["ups"]
    ubar = _complement(ups, n)
    N = np.zeros((n - r, n), np.uint8)
    if n - r:
        N[np.arange(n - r), ubar] = 1
        if r:
            N[:, ups] = res["R"].T
    return N


def solve(A: np.ndarray, p: int, B: np.ndarray):
    """A X = B for the k columns of B (m x k).  With T A = E (Eq. (echelon)),
    A x = b iff E x = T b.  The rows r.. of E are zero, so column b is
    consistent iff (T b)[r:] = K b[rho] + b[rho_bar] is zero; then the
    solution with every non-pivot variable 0 has x[Ups_l] = -(T b)[l] =
    -(M b[rho])[l].  Returns X (n x k, computed for every column; a solution
    where the column is consistent) and a bool per column."""
    A = np.ascontiguousarray(A, dtype=np.uint8)
    B = np.ascontiguousarray(B, dtype=np.uint8)
    m, n = A.shape
    k = B.shape[1]
    res = echelon(A, p)
    r, rho, ups = res["rank"], res["rho"], res["ups"]
    nbar = _complement(rho, m)
    Bp = B[rho].astype(np.int64)
    top = (res["M"].astype(np.int64) @ Bp) % p if r else np.zeros((0, k), np.int64)
    bot = (res["K"].astype(np.int64) @ Bp + B[nbar].astype(np.int64)) % p if m - r else np.zeros((0, k), np.int64)
    X = np.zeros((n, k), np.uint8)
    if r:
        X[ups] = ((-top) % p).astype(np.uint8)
    return X, (bot == 0).all(axis=0)
