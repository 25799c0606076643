"""Thin ctypes binding of libgfe (include/gfe.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; this module
allocates the output / workspace tensors with PyTorch, passes raw device
pointers and the current CUDA stream, and slices the results to the rank.
If libgfe.so is missing the import of a function raises -- there is no
fallback implementation.
"""
from __future__ import annotations

import collections.abc
import contextlib
import ctypes
import os
import threading

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgfe.so")

GFE_U8, GFE_BITS64 = 0, 1
WANT_TRANSFORM, WANT_DENSE_E, WANT_DENSE_T = 0x1, 0x2, 0x4
IMPL_PLAIN, IMPL_TENSOR = 0x100, 0x200
STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "timeout", 4: "busy",
          5: "CUDA error", 6: "internal error", 7: "not supported"}

_i64, _i32, _vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p


class GfeMatrix(ctypes.Structure):
    _fields_ = [("p", _i32), ("m", _i64), ("n", _i64), ("fmt", _i32), ("data", _vp), ("ld", _i64)]


class GfeResult(ctypes.Structure):
    _fields_ = [("rank", _vp), ("pivot_cols", _vp), ("pivot_rows", _vp),
                ("R", _vp), ("ldR", _i64), ("M", _vp), ("ldM", _i64), ("K", _vp), ("ldK", _i64),
                ("E", _vp), ("ldE", _i64), ("T", _vp), ("ldT", _i64)]


class GfeProfile(ctypes.Structure):
    _fields_ = [("launches", _i64 * 8), ("ms", ctypes.c_double * 8), ("madds", ctypes.c_double * 8),
                ("bytes", ctypes.c_double * 8), ("timed", _i64 * 8), ("host_syncs", _i64),
                ("host_wait_ms", ctypes.c_double), ("host_ms", ctypes.c_double)]


class GfeTraceRecord(ctypes.Structure):
    _fields_ = [("kind", _i32), ("clock", _i32), ("m", _i64), ("n", _i64), ("k", _i64), ("stream", ctypes.c_uint64),
                ("start_ms", ctypes.c_double), ("ms", ctypes.c_double)]


KINDS = ["mad_tensor", "mad_plain", "ech_leaf", "rows", "cols", "copy", "convert", "other"]


# every symbol declared in include/gfe.h, with its ctypes signature
SIGNATURES = {
    "gfe_query_workspace": (_i32, [ctypes.POINTER(GfeMatrix), ctypes.c_uint32, ctypes.POINTER(ctypes.c_size_t)]),
    "gfe_query_result_bytes": (_i32, [ctypes.POINTER(GfeMatrix), ctypes.c_uint32, ctypes.POINTER(ctypes.c_size_t)]),
    "gfe_echelon": (_i32, [ctypes.POINTER(GfeMatrix), ctypes.POINTER(GfeResult), ctypes.c_uint32, _vp,
                           ctypes.c_size_t, _vp]),
    "gfe_rank": (_i32, [ctypes.POINTER(GfeMatrix), _vp, _vp, _vp, ctypes.c_uint32, _vp, ctypes.c_size_t, _vp]),
    "gfe_query_batch_workspace": (_i32, [ctypes.POINTER(GfeMatrix), _i32, ctypes.c_uint32,
                                         ctypes.POINTER(ctypes.c_size_t)]),
    "gfe_batch_echelon": (_i32, [ctypes.POINTER(GfeMatrix), ctypes.POINTER(GfeResult), _i32, ctypes.c_uint32,
                                 _vp, ctypes.c_size_t, _vp]),
    "gfe_set_batch_workers": (_i32, [_i32]),
    "gfe_set_wait_policy": (_i32, [_i32]),
    "gfe_set_batch_small_max": (_i32, [_i32, ctypes.c_double]),
    "gfe_set_server_group_work": (_i32, [ctypes.c_double]),
    "gfe_server_create": (_i32, [ctypes.POINTER(_vp), ctypes.c_size_t, _i32, _i32]),
    "gfe_submit": (_i32, [_vp, ctypes.POINTER(GfeMatrix), ctypes.POINTER(GfeResult), ctypes.c_uint32, _vp,
                          ctypes.POINTER(ctypes.c_uint64)]),
    "gfe_poll": (_i32, [_vp, ctypes.c_uint64, ctypes.POINTER(_i32)]),
    "gfe_wait": (_i32, [_vp, ctypes.c_uint64, _i64, ctypes.POINTER(_i32)]),
    "gfe_server_latency": (_i32, [_vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double), _i32]),
    "gfe_server_destroy": (_i32, [_vp]),
    "gfe_mad_workspace": (ctypes.c_size_t, [_i32, _i64, _i64, _i64]),
    "gfe_mad": (_i32, [_i32, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _vp, _i64, ctypes.c_uint32,
                       _vp, ctypes.c_size_t, _vp]),
    "gfe_mad_noalloc_max_bytes": (ctypes.c_size_t, []),
    "gfe_mad_noalloc": (_i32, [_i32, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _vp, _i64, ctypes.c_uint32,
                               _vp]),
    "gfe_nullspace": (_i32, [ctypes.POINTER(GfeMatrix), ctypes.POINTER(GfeResult), _i32, _vp, _i64, _vp]),
    "gfe_solve_workspace": (ctypes.c_size_t, [ctypes.POINTER(GfeMatrix), _i64]),
    "gfe_solve": (_i32, [ctypes.POINTER(GfeMatrix), ctypes.POINTER(GfeResult), _vp, _i64, _i64, _vp, _i64, _vp, _vp,
                         ctypes.c_size_t, _vp]),
    "gfe_mad_gf2": (_i32, [_i64, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _vp]),
    "gfe_gf2_peaks": (_i32, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _vp]),
    "gfe_set_block_policy": (_i32, [_i64, _i64]),
    "gfe_auto_block": (_i64, [_i32, _i64, _i64]),
    "gfe_set_leaf_rows": (_i32, [_i64]),
    "gfe_set_side_tiles": (_i32, [_i32]),
    "gfe_profile_enable": (_i32, [_i32]),
    "gfe_profile_read": (_i32, [ctypes.POINTER(GfeProfile), _i32]),
    "gfe_trace_enable": (_i32, [_i64]),
    "gfe_trace_read": (_i32, [ctypes.POINTER(GfeTraceRecord), _i64, ctypes.POINTER(_i64), _i32]),
    "gfe_selftest_wait_timeout": (_i32, [_i64, _vp]),
    "gfe_status_str": (ctypes.c_char_p, [_i32]),
    "gfe_last_error": (ctypes.c_char_p, []),
    "gfe_version": (ctypes.c_char_p, []),
}

_lib = None


class GfeError(RuntimeError):
    pass


def lib():
    """Load libgfe.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise GfeError("libgfe.so is not built; run paper_1806_04211_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status:
        raise GfeError("%s: %s" % (STATUS.get(status, status), lib().gfe_last_error().decode()))


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t):
    return None if t is None else t.data_ptr()


def words_per_row(n: int) -> int:
    w = (n + 63) // 64
    return w + (w & 1)


def matrix_arg(A: torch.Tensor, p: int, n: int | None = None) -> GfeMatrix:
    """uint8 (m x n) residues, or for p = 2 int64 words (m x ldw) with n given."""
    if A.dtype == torch.uint8:
        m, nn = A.shape
        assert A.numel() == 0 or A.stride(1) == 1
        return GfeMatrix(p, m, nn, GFE_U8, A.data_ptr() if A.numel() else None, max(A.stride(0), nn, 1))
    if A.dtype in (torch.int64,):
        assert p == 2 and n is not None and (A.numel() == 0 or A.stride(1) == 1)
        m = A.shape[0]
        return GfeMatrix(p, m, n, GFE_BITS64, A.data_ptr() if A.numel() else None, 8 * max(A.stride(0), 1))
    raise TypeError("A must be uint8 residues or int64 GF(2) words")


_ws_cache = {}


def _workspace(nbytes: int, device) -> torch.Tensor:
    # one cached workspace per device and host thread: calls made at the same
    # time from several threads must not share one
    key = (str(device), threading.get_ident())
    t = _ws_cache.get(key)
    if t is None or t.numel() < nbytes:
        _ws_cache.pop(key, None)
        t = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device)
        _ws_cache[key] = t
    return t


def release_workspace() -> None:
    """Drop the cached workspace tensors of every thread (the next call
    allocates afresh)."""
    _ws_cache.clear()


def query_workspace(A: torch.Tensor, p: int, n: int | None = None, flags: int = WANT_TRANSFORM) -> int:
    mat = matrix_arg(A, p, n)
    out = ctypes.c_size_t(0)
    _check(lib().gfe_query_workspace(ctypes.byref(mat), flags, ctypes.byref(out)))
    return out.value


def query_result_bytes(A: torch.Tensor, p: int, n: int | None = None, flags: int = WANT_TRANSFORM) -> int:
    """Bytes of the result buffers gfe_echelon writes (gfe_query_result_bytes)."""
    mat = matrix_arg(A, p, n)
    out = ctypes.c_size_t(0)
    _check(lib().gfe_query_result_bytes(ctypes.byref(mat), flags, ctypes.byref(out)))
    return out.value


def _impl_flag(impl: str) -> int:
    return {"tensor": 0, "plain": IMPL_PLAIN}[impl]


def echelon(A: torch.Tensor, p: int, n: int | None = None, transform: bool = True, dense_E: bool = False,
            dense_T: bool = False, impl: str = "tensor", stream=None) -> dict:
    """Echelon form with transformation (gfe_echelon); results on A's device.

    Returns rank (int), rho, ups (int64), R, M, K (and E, T) in A's storage:
    uint8 residues, or for GF(2) int64 bit-packed rows."""
    mat = matrix_arg(A, p, n)
    m, nn = mat.m, mat.n
    mn = min(m, nn)
    dev = A.device
    bits = mat.fmt == GFE_BITS64
    flags = (WANT_TRANSFORM if (transform or dense_T) else 0) | (WANT_DENSE_E if dense_E else 0) | \
        (WANT_DENSE_T if dense_T else 0) | _impl_flag(impl)

    def out(rows, cols):
        if bits:
            return torch.zeros((max(rows, 1), words_per_row(max(cols, 1))), dtype=torch.int64, device=dev)
        return torch.zeros((max(rows, 1), max(cols, 1)), dtype=torch.uint8, device=dev)

    rank = torch.zeros(1, dtype=torch.int64, device=dev)
    pc = torch.zeros(max(mn, 1), dtype=torch.int64, device=dev)
    pr = torch.zeros(max(mn, 1), dtype=torch.int64, device=dev)
    R = out(mn, nn)
    M = out(mn, mn) if transform else None
    K = out(m, mn) if transform else None
    E = out(m, nn) if dense_E else None
    T = out(m, m) if dense_T else None
    es = 8 if bits else 1

    def ld(t):
        return 0 if t is None else t.stride(0) * es

    res = GfeResult(rank.data_ptr(), pc.data_ptr(), pr.data_ptr(), _ptr(R), ld(R), _ptr(M), ld(M), _ptr(K), ld(K),
                    _ptr(E), ld(E), _ptr(T), ld(T))
    need = ctypes.c_size_t(0)
    _check(lib().gfe_query_workspace(ctypes.byref(mat), flags, ctypes.byref(need)))
    ws = _workspace(need.value, dev)
    _check(lib().gfe_echelon(ctypes.byref(mat), ctypes.byref(res), flags, ws.data_ptr(), ws.numel(), _stream(stream)))
    r = int(rank.item())

    def cut(t, rows, cols):
        if t is None:
            return None
        if bits:
            return t[:rows, :words_per_row(cols)] if rows else t[:0]
        return t[:rows, :cols]

    d = dict(rank=r, ups=pc[:r], rho=pr[:r], R=cut(R, r, nn - r))
    if transform:
        d["M"] = cut(M, r, r)
        d["K"] = cut(K, m - r, r)
    if dense_E:
        d["E"] = E[:m]
    if dense_T:
        d["T"] = T[:m]
    return d


def _alloc_result(mat: GfeMatrix, dev, transform: bool):
    m, nn = mat.m, mat.n
    mn = min(m, nn)
    bits = mat.fmt == GFE_BITS64

    def out(rows, cols):
        if bits:
            return torch.zeros((max(rows, 1), words_per_row(max(cols, 1))), dtype=torch.int64, device=dev)
        return torch.zeros((max(rows, 1), max(cols, 1)), dtype=torch.uint8, device=dev)

    bufs = dict(rank=torch.zeros(1, dtype=torch.int64, device=dev),
                ups=torch.zeros(max(mn, 1), dtype=torch.int64, device=dev),
                rho=torch.zeros(max(mn, 1), dtype=torch.int64, device=dev), R=out(mn, nn))
    if transform:
        bufs["M"] = out(mn, mn)
        bufs["K"] = out(m, mn)
    es = 8 if bits else 1

    def ld(t):
        return 0 if t is None else t.stride(0) * es

    res = GfeResult(bufs["rank"].data_ptr(), bufs["ups"].data_ptr(), bufs["rho"].data_ptr(), _ptr(bufs["R"]),
                    ld(bufs["R"]), _ptr(bufs.get("M")), ld(bufs.get("M")), _ptr(bufs.get("K")), ld(bufs.get("K")),
                    None, 0, None, 0)
    return bufs, res


def _cut_result(mat: GfeMatrix, bufs: dict, r: int) -> dict:
    m, nn = mat.m, mat.n
    bits = mat.fmt == GFE_BITS64

    def cut(t, rows, cols):
        if bits:
            return t[:rows, :words_per_row(cols)] if rows else t[:0]
        return t[:rows, :cols]

    d = dict(rank=r, ups=bufs["ups"][:r], rho=bufs["rho"][:r], R=cut(bufs["R"], r, nn - r))
    if "M" in bufs:
        d["M"] = cut(bufs["M"], r, r)
        d["K"] = cut(bufs["K"], m - r, r)
    return d


WAIT_POLICIES = {"auto": 0, "spin": 1, "block": 2}


def set_wait_policy(policy: str) -> None:
    """gfe_set_wait_policy: how the batched form's workers wait ("auto", "spin", "block")."""
    _check(lib().gfe_set_wait_policy(WAIT_POLICIES[policy]))


def set_batch_small_max(side: int = 2048, max_work: float = 0.0) -> None:
    """gfe_set_batch_small_max: largest side (0: none) and work m*n*min(m,n)
    (<= 0: the default) of a batch matrix taken by the one-launch kernel."""
    _check(lib().gfe_set_batch_small_max(side, max_work))


class BatchResult(collections.abc.Mapping):
    """One matrix's result of batch_echelon: the same keys and tensors as
    echelon()'s dict, sliced from the batch's shared buffers when read."""

    __slots__ = ("_bufs", "_mat", "_slots", "_r")

    def __init__(self, bufs, mat, slots, r):
        self._bufs, self._mat, self._slots, self._r = bufs, mat, slots, r

    def __getitem__(self, key):
        if key == "rank":
            return self._r
        r, m, nn = self._r, self._mat.m, self._mat.n
        bits = self._mat.fmt == GFE_BITS64
        if key in ("ups", "rho"):
            off = self._slots["idx"] + 1 + (0 if key == "ups" else self._slots["k"])
            return self._bufs[0][off:off + r]
        if key not in self._slots:
            raise KeyError(key)
        off, rows, cols = self._slots[key]
        t = self._bufs[2 if bits else 1][off:off + rows * cols].view(rows, cols)
        want = {"R": (r, nn - r), "M": (r, r), "K": (m - r, r)}[key]
        if bits:
            return t[:want[0], :words_per_row(want[1])] if want[0] else t[:0]
        return t[:want[0], :want[1]]

    def __iter__(self):
        return iter(["rank", "ups", "rho", "R"] + (["M", "K"] if "M" in self._slots else []))

    def __len__(self):
        return 6 if "M" in self._slots else 4


def _alloc_results(args, dev, transform: bool):
    """Result buffers of a whole batch: three allocations (index arrays, byte
    matrices, GF(2) words; shapes as _alloc_result's), the C structs made
    from their addresses, and each matrix's slots in them."""
    slots, n_idx, n_u8, n_w = [], 0, 0, 0
    for mat in args:
        m, nn = mat.m, mat.n
        k = max(min(m, nn), 1)
        bits = mat.fmt == GFE_BITS64
        sl = {"idx": n_idx, "k": k}
        n_idx += 1 + 2 * k
        shapes = [("R", k, max(nn, 1))] + ([("M", k, k), ("K", max(m, 1), k)] if transform else [])
        for key, rows, cols in shapes:
            if bits:
                cols = words_per_row(cols)
                sl[key] = (n_w, rows, cols)
                n_w += rows * cols
            else:
                sl[key] = (n_u8, rows, cols)
                n_u8 += rows * cols
        slots.append(sl)
    idx = torch.empty(n_idx, dtype=torch.int64, device=dev)
    u8 = torch.empty(n_u8, dtype=torch.uint8, device=dev)
    wb = torch.zeros(n_w, dtype=torch.int64, device=dev)  # rows are padded to whole 16-byte pairs of words
    pi, pu, pw = idx.data_ptr(), u8.data_ptr(), wb.data_ptr()
    res = []
    for mat, sl in zip(args, slots):
        bits = mat.fmt == GFE_BITS64
        base, es = (pw, 8) if bits else (pu, 1)

        def at(key):
            if key not in sl:
                return None, 0
            off, rows, cols = sl[key]
            return base + off * es, cols * es

        R, ldR = at("R")
        M, ldM = at("M")
        K, ldK = at("K")
        o = sl["idx"]
        res.append(GfeResult(pi + 8 * o, pi + 8 * (o + 1), pi + 8 * (o + 1 + sl["k"]), R, ldR, M, ldM, K, ldK,
                             None, 0, None, 0))
    return (idx, u8, wb), slots, res


def batch_echelon(mats, transform: bool = True, impl: str = "tensor", workers: int | None = None, stream=None):
    """gfe_batch_echelon over a list of (A, p) or (A, p, n) tuples; returns a
    list of result mappings.  `workers` applies to this call only (the
    library's worker count returns to its default afterwards)."""
    args = [matrix_arg(*mt) if len(mt) == 3 else matrix_arg(mt[0], mt[1]) for mt in mats]
    if not args:
        return []
    if workers is not None:
        _check(lib().gfe_set_batch_workers(workers))
        try:
            return batch_echelon(mats, transform, impl, None, stream)
        finally:
            lib().gfe_set_batch_workers(0)
    dev = mats[0][0].device
    flags = (WANT_TRANSFORM if transform else 0) | _impl_flag(impl)
    arr = (GfeMatrix * len(args))(*args)
    bufs, slots, res = _alloc_results(args, dev, transform)
    ress = (GfeResult * len(args))(*res)
    need = ctypes.c_size_t(0)
    _check(lib().gfe_query_batch_workspace(arr, len(args), flags, ctypes.byref(need)))
    ws = _workspace(need.value, dev)
    _check(lib().gfe_batch_echelon(arr, ress, len(args), flags, ws.data_ptr(), ws.numel(), _stream(stream)))
    with torch.cuda.stream(stream) if stream is not None else contextlib.nullcontext():
        ranks = bufs[0][torch.tensor([sl["idx"] for sl in slots], device=dev)].cpu().tolist()
    return [BatchResult(bufs, a, sl, int(r)) for a, sl, r in zip(args, slots, ranks)]


def rank(A: torch.Tensor, p: int, n: int | None = None, impl: str = "tensor", stream=None) -> dict:
    """Rank and pivots only (gfe_rank)."""
    mat = matrix_arg(A, p, n)
    mn = min(mat.m, mat.n)
    dev = A.device
    rk = torch.zeros(1, dtype=torch.int64, device=dev)
    pc = torch.zeros(max(mn, 1), dtype=torch.int64, device=dev)
    pr = torch.zeros(max(mn, 1), dtype=torch.int64, device=dev)
    need = ctypes.c_size_t(0)
    _check(lib().gfe_query_workspace(ctypes.byref(mat), 0, ctypes.byref(need)))
    ws = _workspace(need.value, dev)
    _check(lib().gfe_rank(ctypes.byref(mat), rk.data_ptr(), pc.data_ptr(), pr.data_ptr(), _impl_flag(impl),
                          ws.data_ptr(), ws.numel(), _stream(stream)))
    r = int(rk.item())
    return dict(rank=r, ups=pc[:r], rho=pr[:r])


def _result_struct(res, dev, bits: bool):
    """A gfe_result of device pointers for an echelon() / batch_echelon()
    result mapping (the rank goes to the device as an int64 scalar)."""
    es = 8 if bits else 1
    rk = torch.tensor([int(res["rank"])], dtype=torch.int64, device=dev)

    def addr(t):
        # the address of the view's first element, also for an empty view
        # (the result tensors are views of buffers of at least one row)
        return t.untyped_storage().data_ptr() + t.storage_offset() * t.element_size()

    def p_ld(key):
        t = res[key] if key in res else None
        return (None, 0) if t is None else (addr(t), t.stride(0) * es)

    R, ldR = p_ld("R")
    M, ldM = p_ld("M")
    K, ldK = p_ld("K")
    ups = res["ups"]
    rho = res["rho"]
    keep = (rk, ups, rho)
    st = GfeResult(rk.data_ptr(), addr(ups), addr(rho), R, ldR, M, ldM, K, ldK, None, 0, None, 0)
    return st, keep


def _shape_arg(p: int, m: int, n: int, bits: bool) -> GfeMatrix:
    return GfeMatrix(p, m, n, GFE_BITS64 if bits else GFE_U8, None, 8 * words_per_row(max(n, 1)) if bits else max(n, 1))


def nullspace(res, p: int, m: int, n: int, side: str = "right", bits: bool | None = None, stream=None) -> torch.Tensor:
    """gfe_nullspace: basis of the left ({y : y A = 0}, rows of (K 1) P_rho)
    or right ({x : A x = 0}) null space of the matrix `res` was computed for,
    one basis vector per row, in A's storage (uint8, or GF(2) words)."""
    r = int(res["rank"])
    dev = res["ups"].device
    bits = (p == 2 and res["R"].dtype == torch.int64) if bits is None else bits
    length = m if side == "left" else n
    rows = length - r
    if bits:
        N = torch.zeros((max(length, 1), words_per_row(max(length, 1))), dtype=torch.int64, device=dev)
    else:
        N = torch.zeros((max(length, 1), max(length, 1)), dtype=torch.uint8, device=dev)
    st, keep = _result_struct(res, dev, bits)
    mat = _shape_arg(p, m, n, bits)
    _check(lib().gfe_nullspace(ctypes.byref(mat), ctypes.byref(st), 0 if side == "left" else 1, N.data_ptr(),
                               N.stride(0) * (8 if bits else 1), _stream(stream)))
    if bits:
        return N[:rows, :words_per_row(length)] if rows else N[:0]
    return N[:rows, :length]


def solve(res, p: int, m: int, n: int, B: torch.Tensor, k: int | None = None, stream=None):
    """gfe_solve: X (n x k) with A X = B where consistent, and the int32
    consistency flag per column.  B is m x k uint8, or for GF(2) bit rows
    (int64 words, k given)."""
    dev = B.device
    bits = B.dtype == torch.int64
    if k is None:
        k = B.shape[1]
    if bits:
        X = torch.zeros((max(n, 1), words_per_row(max(k, 1))), dtype=torch.int64, device=dev)
    else:
        X = torch.zeros((max(n, 1), max(k, 1)), dtype=torch.uint8, device=dev)
    ok = torch.zeros(max(k, 1), dtype=torch.int32, device=dev)
    st, keep = _result_struct(res, dev, bits)
    mat = _shape_arg(p, m, n, bits)
    need = lib().gfe_solve_workspace(ctypes.byref(mat), k)
    ws = _workspace(need, dev)
    es = 8 if bits else 1
    _check(lib().gfe_solve(ctypes.byref(mat), ctypes.byref(st), B.data_ptr() if B.numel() else None,
                           B.stride(0) * es if B.numel() else 0, k, X.data_ptr(), X.stride(0) * es, ok.data_ptr(),
                           ws.data_ptr(), ws.numel(), _stream(stream)))
    return X[:n], ok[:k]


def mad(W, A: torch.Tensor, B: torch.Tensor, p: int, impl: str = "tensor", out=None, stream=None) -> torch.Tensor:
    """C := W + A B over GF(p) on uint8 residues (gfe_mad); W may be None."""
    m, k = A.shape
    n = B.shape[1]
    C = out if out is not None else torch.empty((m, n), dtype=torch.uint8, device=A.device)
    need = lib().gfe_mad_workspace(p, m, n, k)
    ws = _workspace(need, A.device)
    _check(lib().gfe_mad(p, m, n, k, _ptr(W), W.stride(0) if W is not None else 0, _ptr(A), A.stride(0), _ptr(B),
                         B.stride(0), C.data_ptr(), C.stride(0), _impl_flag(impl), ws.data_ptr(), ws.numel(),
                         _stream(stream)))
    return C


def mad_gf2(W, A: torch.Tensor, B: torch.Tensor, n: int, k: int, out=None, stream=None) -> torch.Tensor:
    """gfe_mad_gf2: C := W + A B over GF(2) on bit-packed int64 rows (A m x k
    bits, B k x n bits, W and C m x n bits); W may be None or `out`."""
    m = A.shape[0]
    C = out if out is not None else torch.zeros((m, words_per_row(max(n, 1))), dtype=torch.int64, device=A.device)
    _check(lib().gfe_mad_gf2(m, n, k, _ptr(W), 8 * W.stride(0) if W is not None else 0, _ptr(A), 8 * A.stride(0),
                             _ptr(B), 8 * B.stride(0), C.data_ptr(), 8 * C.stride(0), _stream(stream)))
    return C


def gf2_peaks(stream=None) -> dict:
    """gfe_gf2_peaks: measured LOP3 rate and 128-bit shared-memory load rate."""
    a, b = ctypes.c_double(0), ctypes.c_double(0)
    _check(lib().gfe_gf2_peaks(ctypes.byref(a), ctypes.byref(b), _stream(stream)))
    return {"lop3_per_s": a.value, "lds_bytes_per_s": b.value, "gf2_madds_per_s_alu": 32.0 * a.value}


def mad_noalloc(W, A: torch.Tensor, B: torch.Tensor, p: int, out: torch.Tensor, impl: str = "tensor", stream=None):
    """gfe_mad_noalloc: C := W + A B over GF(p) into `out` without any device
    allocation by the library (its scratch is a fixed library-owned array)."""
    m, k = A.shape
    n = B.shape[1]
    _check(lib().gfe_mad_noalloc(p, m, n, k, _ptr(W), W.stride(0) if W is not None else 0, _ptr(A), A.stride(0),
                                 _ptr(B), B.stride(0), out.data_ptr(), out.stride(0), _impl_flag(impl),
                                 _stream(stream)))
    return out


def set_block_policy(threshold: int = 0, block: int = 0):
    """Block partition policy (gfe_set_block_policy); 0, 0 = the measured
    table (gfe_auto_block)."""
    _check(lib().gfe_set_block_policy(threshold, block))


def set_leaf_rows(rows: int = 0):
    """Rows of a leaf block in the planner's leaf grid (gfe_set_leaf_rows); 0 = default."""
    _check(lib().gfe_set_leaf_rows(rows))


def auto_block(p: int, m: int, n: int) -> int:
    """Block side the default policy uses for an m x n matrix over GF(p)."""
    return int(lib().gfe_auto_block(p, m, n))


def autotune_block(p: int, m: int, n: int, candidates=(2048, 3072, 4096), rank=None, device="cuda:0",
                   reps: int = 2, seed: int = 1) -> dict:
    """Times gfe_echelon on a seeded synthetic m x n matrix over GF(p) (rank
    `rank`, None = uniform) with each candidate block side, sets the fastest
    with gfe_set_block_policy and returns {side: seconds}."""
    import time
    from . import synth
    A = synth.matrix(p, m, n, seed=seed, rank=rank, device=device)
    kw = dict(n=n) if p == 2 else {}
    times = {}
    for blk in candidates:
        set_block_policy(blk, blk)
        echelon(A, p, **kw)
        torch.cuda.synchronize(device)
        best = float("inf")
        for _ in range(reps):
            t0 = time.perf_counter()
            echelon(A, p, **kw)
            torch.cuda.synchronize(device)
            best = min(best, time.perf_counter() - t0)
        times[blk] = best
    winner = min(times, key=times.get)
    set_block_policy(winner, winner)
    return times


def profile_enable(on: bool = True, kinds=None):
    """Count every launch; time (CUDA events) the given kinds (default all)."""
    mask = 0
    if on:
        mask = -1 if kinds is None else sum(1 << KINDS.index(k) for k in kinds)
    _check(lib().gfe_profile_enable(mask))


def profile_read(reset: bool = True) -> dict:
    pr = GfeProfile()
    _check(lib().gfe_profile_read(ctypes.byref(pr), 1 if reset else 0))
    return dict(launches={k: pr.launches[i] for i, k in enumerate(KINDS)},
                ms={k: pr.ms[i] for i, k in enumerate(KINDS)},
                madds={k: pr.madds[i] for i, k in enumerate(KINDS)},
                bytes={k: pr.bytes[i] for i, k in enumerate(KINDS)},
                timed={k: pr.timed[i] for i, k in enumerate(KINDS)},
                host_syncs=pr.host_syncs, host_wait_ms=pr.host_wait_ms, host_ms=pr.host_ms)


def trace_enable(capacity: int = 1 << 20):
    """Keep a per-launch record (kind, shape, stream, start, duration) of up
    to `capacity` timed launches (gfe_trace_enable); 0 stops and drops them.
    Records are made only while the profile is enabled."""
    _check(lib().gfe_trace_enable(capacity))


def trace_read(reset: bool = True) -> list:
    n = ctypes.c_int64(0)
    _check(lib().gfe_trace_read(None, 0, ctypes.byref(n), 0))
    buf = (GfeTraceRecord * max(n.value, 1))()
    _check(lib().gfe_trace_read(buf, n.value, ctypes.byref(n), 1 if reset else 0))
    return [dict(kind=KINDS[r.kind], clock=("event", "device")[r.clock], m=r.m, n=r.n, k=r.k, stream=r.stream,
                 start_ms=r.start_ms, ms=r.ms) for r in buf[:n.value]]


class Server:
    """gfe_server: continuous-batching echelonisation service (C ABI)."""

    def __init__(self, hbm_cap_bytes: int, workers: int = 8, device: int = 0):
        self._h = _vp()
        _check(lib().gfe_server_create(ctypes.byref(self._h), hbm_cap_bytes, workers, device))
        self._pending = {}

    def submit(self, A: torch.Tensor, p: int, n: int | None = None, transform: bool = True, impl: str = "tensor",
               stream=None) -> int:
        mat = matrix_arg(A, p, n)
        bufs, res = _alloc_result(mat, A.device, transform)
        flags = (WANT_TRANSFORM if transform else 0) | _impl_flag(impl)
        t = ctypes.c_uint64(0)
        _check(lib().gfe_submit(self._h, ctypes.byref(mat), ctypes.byref(res), flags, _stream(stream),
                                ctypes.byref(t)))
        self._pending[t.value] = (A, mat, bufs, res)
        return t.value

    def poll(self, ticket: int) -> bool:
        st = _i32(0)
        rc = lib().gfe_poll(self._h, ticket, ctypes.byref(st))
        if rc == 4:
            return False
        _check(rc)
        _check(st.value)
        return True

    def wait(self, ticket: int, timeout_us: int = -1) -> dict:
        """Result of a request (and its submit-to-done latency in us)."""
        st = _i32(0)
        _check(lib().gfe_wait(self._h, ticket, timeout_us, ctypes.byref(st)))
        _check(st.value)
        us = ctypes.c_double(0)
        _check(lib().gfe_server_latency(self._h, ticket, ctypes.byref(us), 1))
        A, mat, bufs, res = self._pending.pop(ticket)
        d = _cut_result(mat, bufs, int(bufs["rank"].item()))
        d["latency_us"] = us.value
        return d

    def close(self):
        if self._h:
            _check(lib().gfe_server_destroy(self._h))
            self._h = _vp()
            self._pending.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
