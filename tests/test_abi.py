"""The C-ABI library builds, loads and exports every symbol include/gfe.h
declares; host-side argument checks and workspace planning (no GPU needed)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT
from paper_1806_04211_gb300 import build, gfe


def header_functions():
    src = open(os.path.join(ROOT, "include", "gfe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gfe_[a-z0-9_]+)\s*\(", src)))


def test_build_and_load():
    path = build.build()
    assert os.path.exists(path)
    assert gfe.lib().gfe_version().startswith(b"gfe")


def test_every_declared_symbol_is_exported():
    L = gfe.lib()
    names = header_functions()
    assert "gfe_echelon" in names and "gfe_rank" in names and "gfe_mad" in names
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(gfe.SIGNATURES), set(names) ^ set(gfe.SIGNATURES)


def query(p, m, n, fmt=0, ld=None, flags=1):
    mat = gfe.GfeMatrix(p, m, n, fmt, 1, ld if ld is not None else n)
    out = ctypes.c_size_t(0)
    st = gfe.lib().gfe_query_workspace(ctypes.byref(mat), flags, ctypes.byref(out))
    return st, out.value


@pytest.mark.parametrize("p", [4, 1, 0, 253, 256, -3])
def test_rejects_non_prime_or_large_p(p):
    st, _ = query(p, 10, 10)
    assert st == 1
    assert b"prime" in gfe.lib().gfe_last_error()


def test_rejects_bad_shapes_and_formats():
    assert query(3, -1, 5)[0] == 1
    assert query(3, 5, 10, ld=9)[0] == 1
    assert query(3, 5, 10, fmt=1, ld=16)[0] == 1        # BITS64 needs p = 2
    assert query(2, 5, 130, fmt=1, ld=16)[0] == 1       # 130 bits need 3 words
    assert query(2, 5, 130, fmt=1, ld=20)[0] == 1       # not a multiple of 8
    assert query(2, 5, 130, fmt=1, ld=24)[0] == 0
    assert query(3, 5, 10, fmt=7)[0] == 1


def test_workspace_monotone_and_empty():
    assert query(3, 0, 0)[0] == 0
    assert query(3, 0, 7)[0] == 0
    prev = 0
    for n in (10, 100, 1000, 5000, 9000, 20000):
        st, ws = query(7, n, n)
        assert st == 0 and ws >= prev
        prev = ws
    # the internal copy of the input alone takes 2 bytes (bf16) per entry
    assert query(251, 4000, 4000)[1] > 2 * 4000 * 4000


def test_null_result_rejected():
    mat = gfe.GfeMatrix(3, 4, 4, 0, 1, 4)
    st = gfe.lib().gfe_echelon(ctypes.byref(mat), None, 1, None, 0, None)
    assert st == 1


def test_status_strings():
    L = gfe.lib()
    assert L.gfe_status_str(0) == b"ok"
    assert L.gfe_status_str(1) == b"invalid argument"


def test_block_policy_validation():
    """A block wider than the threshold would recurse without end."""
    for thr, blk in [(1024, 2048), (100, 200)]:
        with pytest.raises(gfe.GfeError):
            gfe.set_block_policy(thr, blk)
    gfe.set_block_policy(4096, 4096)
    gfe.set_block_policy(40, 16)
    gfe.set_block_policy(3072, 0)   # one side given: the other takes its value
    gfe.set_block_policy()


def test_wait_policy_validation():
    for bad in (-1, 3):
        with pytest.raises(gfe.GfeError):
            gfe._check(gfe.lib().gfe_set_wait_policy(bad))
    for name in ("spin", "block", "auto"):
        gfe.set_wait_policy(name)


def test_auto_block_table():
    """The default policy's measured table: GF(2) grows with the size, larger
    fields keep 2048; every side is a multiple of the 1024-row leaf."""
    assert gfe.auto_block(2, 8192, 8192) == 2048
    assert gfe.auto_block(2, 32768, 32768) == 3072
    assert gfe.auto_block(2, 100000, 100000) == 6144
    assert gfe.auto_block(7, 32768, 32768) == 2048
    assert gfe.auto_block(251, 20000, 50000) == 1024
    assert gfe.auto_block(13, 20000, 20000) == 2048
    for p in (2, 3, 251):
        for n in (100, 5000, 20000, 70000, 200000):
            assert gfe.auto_block(p, n, n) % 1024 == 0


def test_batch_small_policy_validation():
    with pytest.raises(gfe.GfeError):
        gfe._check(gfe.lib().gfe_set_batch_small_max(-1, 0.0))
    gfe.set_batch_small_max(512, 1e8)
    gfe.set_batch_small_max()


def test_solve_nullspace_and_gf2_mad_reject_bad_arguments():
    """Argument checks that return before any CUDA call."""
    L = gfe.lib()
    mat = gfe.GfeMatrix(7, 10, 8, 0, None, 8)
    rk = ctypes.c_int64(0)
    res = gfe.GfeResult(ctypes.addressof(rk), 1, 1, 1, 8, 1, 8, 1, 8, None, 0, None, 0)
    assert L.gfe_nullspace(ctypes.byref(mat), ctypes.byref(res), 5, 1, 16, None) == 1  # bad side
    assert b"side" in L.gfe_last_error()
    bad = gfe.GfeMatrix(4, 10, 8, 0, None, 8)  # 4 is not prime
    assert L.gfe_nullspace(ctypes.byref(bad), ctypes.byref(res), 0, 1, 16, None) == 1
    bits3 = gfe.GfeMatrix(3, 10, 8, 1, None, 8)  # GFE_BITS64 needs p = 2
    assert L.gfe_nullspace(ctypes.byref(bits3), ctypes.byref(res), 0, 1, 16, None) == 1
    assert L.gfe_nullspace(ctypes.byref(mat), ctypes.byref(res), 0, 1, 4, None) == 1  # ldn < m
    assert L.gfe_solve_workspace(ctypes.byref(mat), -1) == 0
    assert L.gfe_solve_workspace(ctypes.byref(mat), 3) > 0
    assert L.gfe_solve(ctypes.byref(mat), ctypes.byref(res), 1, 8, -1, 1, 8, 1, 1, 1 << 20, None) == 1
    assert L.gfe_solve(ctypes.byref(mat), ctypes.byref(res), 1, 8, 0, 1, 8, 1, 1, 1 << 20, None) == 0  # k = 0
    assert L.gfe_solve(ctypes.byref(mat), ctypes.byref(res), 1, 8, 3, 1, 8, None, 1, 1 << 20, None) == 1
    assert L.gfe_solve(ctypes.byref(mat), ctypes.byref(res), 1, 8, 3, 1, 8, 1, 1, 16, None) == 1  # small ws
    assert b"workspace" in L.gfe_last_error()
    # packed GF(2) multiply-add: pitches must be whole words covering a row
    assert L.gfe_mad_gf2(4, 100, 70, None, 0, 1, 16, 1, 12, 1, 16, None) == 1
    assert L.gfe_mad_gf2(4, 100, 70, None, 0, 1, 8, 1, 16, 1, 16, None) == 1
    assert L.gfe_mad_gf2(-1, 100, 70, None, 0, 1, 16, 1, 16, 1, 16, None) == 1
    assert L.gfe_mad_gf2(0, 100, 70, None, 0, 1, 16, 1, 16, 1, 16, None) == 0  # empty: nothing to do
    assert L.gfe_set_side_tiles(-1) == 1 and L.gfe_set_side_tiles(2000) == 1
    assert L.gfe_set_side_tiles(4) == 0


def test_query_result_bytes():
    """gfe_query_result_bytes: the worst-case result buffers, 256-byte rounded,
    computed on the host."""
    L = gfe.lib()

    def q(p, m, n, flags, fmt=0, ld=None):
        mat = gfe.GfeMatrix(p, m, n, fmt, 64, ld if ld is not None else (((n + 63) // 64) * 8 if fmt else n))
        out = ctypes.c_size_t(0)
        assert L.gfe_query_result_bytes(ctypes.byref(mat), flags, ctypes.byref(out)) == 0, L.gfe_last_error()
        return out.value

    a = lambda x: (x + 255) // 256 * 256
    m, n, k = 300, 200, 200
    base = a(8) + 2 * a(8 * k) + a(k * n)
    assert q(7, m, n, 0) == base
    assert q(7, m, n, 1) == base + a(k * k) + a(m * k)
    assert q(7, m, n, 1 | 2 | 4) == base + a(k * k) + a(m * k) + a(m * n) + a(m * m)
    assert q(7, m, n, 4) == base + a(k * k) + a(m * k) + a(m * m)  # dense T needs M and K
    words = lambda c: (c + 63) // 64 * 8
    assert q(2, m, n, 1, fmt=1) == a(8) + 2 * a(8 * k) + a(k * words(n)) + a(k * words(k)) + a(m * words(k))
    assert q(3, 0, 5, 1) == a(8) + 2 * a(0) + a(0) + a(0) + a(0)
    # bad arguments: rejected before anything else
    mat = gfe.GfeMatrix(4, 3, 3, 0, 64, 3)
    out = ctypes.c_size_t(0)
    assert L.gfe_query_result_bytes(ctypes.byref(mat), 1, ctypes.byref(out)) == 1
    mat = gfe.GfeMatrix(7, 3, 3, 0, 64, 3)
    assert L.gfe_query_result_bytes(ctypes.byref(mat), 1, None) == 1
