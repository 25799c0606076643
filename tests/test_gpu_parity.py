"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by
element, on seeded inputs (GPU)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1806_04211_gb300 import gfe, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def compare_u8(A, p, got, ref):
    assert got["rank"] == ref["rank"]
    r = ref["rank"]
    for k in ("rho", "ups"):
        assert np.array_equal(got[k].cpu().numpy(), ref[k]), k
    for k in ("R", "M", "K"):
        if k not in got:
            continue
        g = got[k].cpu().numpy()
        assert g.shape == ref[k].shape, (k, g.shape, ref[k].shape)
        assert np.array_equal(g, ref[k]), (k, np.argwhere(g != ref[k])[:5])


def compare_gf2(got, ref, m, n):
    assert got["rank"] == ref["rank"]
    r = ref["rank"]
    for k in ("rho", "ups"):
        assert np.array_equal(got[k].cpu().numpy(), ref[k]), k
    for k, cols in (("R", n - r), ("M", r), ("K", r)):
        if k not in got:
            continue
        g = O.unpack_bits(got[k].cpu().numpy(), cols) if got[k].numel() else np.zeros((0, cols), np.uint8)
        e = O.unpack_bits(ref[k], cols) if ref[k].size else np.zeros((0, cols), np.uint8)
        rows = e.shape[0]
        assert np.array_equal(g[:rows], e), k


@pytest.fixture(autouse=True)
def _policy():
    gfe.set_block_policy()
    yield
    gfe.set_block_policy()


CASES = [
    # p, m, n, rank (None = uniform)
    (3, 1, 1, None), (3, 7, 5, None), (3, 64, 64, None), (3, 65, 63, None),
    (3, 300, 200, None), (5, 257, 513, None), (7, 1500, 700, None), (7, 700, 1500, 300),
    (3, 1000, 1000, None), (3, 1000, 1000, 700), (31, 333, 444, None),
    (37, 200, 300, None), (251, 400, 400, None), (251, 600, 450, 270), (193, 129, 1100, None),
    (11, 300, 200, None), (13, 200, 300, 150), (5, 1100, 130, None), (13, 1030, 64, None),
]


@pytest.mark.parametrize("impl", ["tensor", "plain"])
@pytest.mark.parametrize("p,m,n,rank", CASES)
def test_parity_u8(p, m, n, rank, impl):
    A = synth.matrix(p, m, n, seed=3, rank=rank)
    ref = O.echelon(A.numpy(), p)
    got = gfe.echelon(A.to(DEV), p, impl=impl)
    compare_u8(A, p, got, ref)


@pytest.mark.parametrize("m,n,rank", [(1, 1, None), (64, 64, None), (100, 130, None), (1030, 500, None),
                                      (700, 1200, 500), (2000, 2000, None)])
def test_parity_gf2(m, n, rank):
    A = synth.matrix(2, m, n, seed=5, rank=rank)
    ref = O.echelon_gf2(A.numpy(), m, n)
    got = gfe.echelon(A.to(DEV), 2, n=n)
    compare_gf2(got, ref, m, n)


@pytest.mark.parametrize("p,m,n,rank", [(3, 700, 500, None), (7, 600, 900, 400), (251, 300, 350, 200),
                                        (2, 600, 700, None)])
def test_parity_recursive_chief(p, m, n, rank):
    """Small block policy: the top-level Chief uses 128-square blocks whose
    ECH is itself a Chief over leaf blocks (the recursive scheme)."""
    gfe.set_block_policy(200, 128)
    A = synth.matrix(p, m, n, seed=9, rank=rank)
    if p == 2:
        ref = O.echelon_gf2(A.numpy(), m, n)
        compare_gf2(gfe.echelon(A.to(DEV), 2, n=n), ref, m, n)
    else:
        ref = O.echelon(A.numpy(), p)
        compare_u8(A, p, gfe.echelon(A.to(DEV), p), ref)


@pytest.mark.parametrize("p,m,n,rank,blk", [(2, 4000, 7000, None, 3072), (2, 7000, 3500, 2500, 3072),
                                            (7, 3300, 700, None, 3072)])
def test_parity_block_3072(p, m, n, rank, blk):
    """The 3072-wide top-level blocks the default policy picks for large GF(2)
    inputs (three leaf row blocks per block), on sizes the oracle finishes."""
    gfe.set_block_policy(blk, blk)
    A = synth.matrix(p, m, n, seed=12, rank=rank)
    if p == 2:
        ref = O.echelon_gf2(A.numpy(), m, n)
        compare_gf2(gfe.echelon(A.to(DEV), 2, n=n), ref, m, n)
    else:
        ref = O.echelon(A.numpy(), p)
        compare_u8(A, p, gfe.echelon(A.to(DEV), p), ref)


@pytest.mark.parametrize("p,m,n,rank,blk", [(251, 700, 3000, 100, 512), (7, 1500, 4000, 300, 1024),
                                            (2, 3000, 6000, 500, 1024), (31, 900, 2500, 0, 512)])
def test_parity_zero_blocks(p, m, n, rank, blk):
    """Wide rank-deficient inputs (rank 0 included): past the rank whole row
    blocks are zero and are skipped after one zero test; the fp32 leaf
    (p > 13) and nested Chiefs over leaves are exercised."""
    gfe.set_block_policy(blk, blk)
    A = synth.matrix(p, m, n, seed=15, rank=rank) if rank else torch.zeros((m, n), dtype=torch.uint8)
    if p == 2:
        A = synth.matrix(p, m, n, seed=15, rank=rank)
        ref = O.echelon_gf2(A.numpy(), m, n)
        compare_gf2(gfe.echelon(A.to(DEV), 2, n=n), ref, m, n)
    else:
        ref = O.echelon(A.numpy(), p)
        compare_u8(A, p, gfe.echelon(A.to(DEV), p), ref)


@pytest.mark.parametrize("p,m,n,leaf_rows", [(3, 900, 300, 256), (2, 1500, 700, 128), (251, 700, 200, 512)])
def test_parity_leaf_rows(p, m, n, leaf_rows):
    """Shorter leaf row blocks (gfe_set_leaf_rows) change the block grid, not
    the result."""
    gfe.set_leaf_rows(leaf_rows)
    try:
        A = synth.matrix(p, m, n, seed=13)
        if p == 2:
            ref = O.echelon_gf2(A.numpy(), m, n)
            compare_gf2(gfe.echelon(A.to(DEV), 2, n=n), ref, m, n)
        else:
            ref = O.echelon(A.numpy(), p)
            compare_u8(A, p, gfe.echelon(A.to(DEV), p), ref)
    finally:
        gfe.set_leaf_rows(0)


def test_autotune_block_sets_a_candidate():
    """The autotuner times every candidate and leaves the fastest in force;
    results do not depend on the policy it picks."""
    times = gfe.autotune_block(2, 3000, 3000, candidates=(1024, 2048), reps=1)
    assert sorted(times) == [1024, 2048] and all(t > 0 for t in times.values())
    A = synth.matrix(2, 1200, 900, seed=14)
    ref = O.echelon_gf2(A.numpy(), 1200, 900)
    compare_gf2(gfe.echelon(A.to(DEV), 2, n=900), ref, 1200, 900)
    gfe.set_block_policy()


@pytest.mark.parametrize("p", [3, 251])
def test_dense_E_T(p):
    A = synth.matrix(p, 150, 170, seed=2, rank=100)
    ref = O.echelon(A.numpy(), p, want_E=True, want_T=True)
    got = gfe.echelon(A.to(DEV), p, dense_E=True, dense_T=True)
    assert np.array_equal(got["E"].cpu().numpy(), ref["E"])
    assert np.array_equal(got["T"].cpu().numpy(), ref["T"])


def test_dense_E_T_gf2():
    m, n = 140, 200
    A = synth.matrix(2, m, n, seed=2)
    ref = O.echelon_gf2(A.numpy(), m, n, want_E=True, want_T=True)
    got = gfe.echelon(A.to(DEV), 2, n=n, dense_E=True, dense_T=True)
    assert np.array_equal(O.unpack_bits(got["E"].cpu().numpy(), n), O.unpack_bits(ref["E"], n))
    assert np.array_equal(O.unpack_bits(got["T"].cpu().numpy(), m), O.unpack_bits(ref["T"], m))


@pytest.mark.parametrize("p", [2, 3, 7, 251])
def test_edge_cases(p):
    for A in [np.zeros((5, 7), np.uint8), np.eye(9, dtype=np.uint8), np.zeros((0, 4), np.uint8),
              np.zeros((4, 0), np.uint8), np.ones((6, 6), np.uint8),
              np.tile(np.arange(5, dtype=np.uint8) % p, (4, 1))]:
        ref = O.echelon(A, p)
        got = gfe.echelon(torch.from_numpy(A).to(DEV), p)
        compare_u8(A, p, got, ref)


def test_duplicate_rows_and_zero_columns():
    p = 5
    A = synth.uniform_u8(300, 200, p, seed=4).numpy()
    A[150] = A[3]
    A[:, 40] = 0
    A[:, 41] = A[:, 7]
    ref = O.echelon(A, p)
    compare_u8(A, p, gfe.echelon(torch.from_numpy(A).to(DEV), p), ref)


@pytest.mark.parametrize("p", [3, 7, 251])
def test_rank_only(p):
    A = synth.matrix(p, 500, 400, seed=6, rank=250)
    ref = O.echelon(A.numpy(), p)
    got = gfe.rank(A.to(DEV), p)
    assert got["rank"] == ref["rank"]
    assert np.array_equal(got["rho"].cpu().numpy(), ref["rho"])
    assert np.array_equal(got["ups"].cpu().numpy(), ref["ups"])


@pytest.mark.parametrize("impl", ["tensor", "plain"])
@pytest.mark.parametrize("p,m,n,k", [(2, 200, 300, 100), (3, 129, 257, 513), (7, 300, 300, 4096),
                                     (31, 64, 64, 64), (251, 200, 190, 1500), (251, 1, 1, 1)])
def test_mad(p, m, n, k, impl):
    W = synth.uniform_u8(m, n, p, 1, 0)
    A = synth.uniform_u8(m, k, p, 1, 1)
    B = synth.uniform_u8(k, n, p, 1, 2)
    ref = (W.numpy().astype(np.int64) + A.numpy().astype(np.int64) @ B.numpy().astype(np.int64)) % p
    got = gfe.mad(W.to(DEV), A.to(DEV), B.to(DEV), p, impl=impl).cpu().numpy()
    assert np.array_equal(got, ref)
    got0 = gfe.mad(None, A.to(DEV), B.to(DEV), p, impl=impl).cpu().numpy()
    assert np.array_equal(got0, (A.numpy().astype(np.int64) @ B.numpy().astype(np.int64)) % p)


def _kchunk(p):
    if p == 2:  # parity read from the mantissa of (sum + 2^23): sums stay below 2^22
        return (1 << 22) // 64 * 64
    cmax = (p - 1) // 2
    return ((1 << 24) - 1) // (cmax * cmax) // 64 * 64


@pytest.mark.parametrize("p", [2, 3, 7, 31, 37, 251])
def test_mad_tensor_exact_at_the_accumulation_bound(p):
    """Every product at the largest centred magnitude and of one sign per
    column, with K just past the exact-accumulation chunk (capped at 2^20 for
    p <= 3): the fp32 partial sums come within one chunk of 2^24 (2^20).  The
    expected value is the closed form K * (+-cmax^2) + W mod p."""
    cmax = 1 if p == 2 else (p - 1) // 2
    k = min(_kchunk(p) + 200, 1 << 20) if p != 2 else _kchunk(p) + 200
    m, n = 8, 40
    A = torch.full((m, k), cmax, dtype=torch.uint8, device=DEV)
    B = torch.full((k, n), cmax, dtype=torch.uint8, device=DEV)
    B[:, 1::2] = (p - cmax) % p                        # -cmax in odd columns
    W = synth.uniform_u8(m, n, p, 2, 0)
    sign = np.where(np.arange(n) % 2 == 0, 1, -1)
    ref = (W.numpy().astype(np.int64) + (k * cmax * cmax) * sign[None, :]) % p
    gfe.profile_enable(True)
    gfe.profile_read(True)
    got = gfe.mad(W.to(DEV), A, B, p, impl="tensor").cpu().numpy()
    prof = gfe.profile_read(True)
    gfe.profile_enable(False)
    assert prof["launches"]["mad_tensor"] >= 1 and prof["launches"]["mad_plain"] == 0
    assert np.array_equal(got, ref)


def test_tensor_path_is_taken_in_echelon():
    p, n = 7, 3000
    A = synth.matrix(p, n, n, seed=8, rank=2000)
    gfe.profile_enable(True)
    gfe.profile_read(True)
    got = gfe.echelon(A.to(DEV), p)
    prof = gfe.profile_read(True)
    gfe.profile_enable(False)
    assert got["rank"] == 2000
    assert prof["launches"]["mad_tensor"] > 0
    assert prof["madds"]["mad_tensor"] > 10 * prof["madds"]["mad_plain"]


@pytest.mark.parametrize("p,m,n,rank", [(2, 4200, 3000, None), (2, 2049, 5000, 1500), (3, 2100, 1400, None),
                                        (251, 2300, 1100, 700), (7, 1100, 2300, None)])
def test_parity_default_policy_ragged_top_blocks(p, m, n, rank):
    """Sizes past the default 2048 threshold: 2048-square top-level blocks
    with ragged last blocks, each ECH a Chief over leaf blocks."""
    A = synth.matrix(p, m, n, seed=21, rank=rank)
    if p == 2:
        ref = O.echelon_gf2(A.numpy(), m, n)
        compare_gf2(gfe.echelon(A.to(DEV), 2, n=n), ref, m, n)
    else:
        ref = O.echelon(A.numpy(), p)
        compare_u8(A, p, gfe.echelon(A.to(DEV), p), ref)
