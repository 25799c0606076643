"""Solving and null spaces from the echelon result (gfe_solve, gfe_nullspace)
against the oracle, element by element, on seeded inputs (GPU)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1806_04211_gb300 import gfe, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

CASES = [
    # p, m, n, rank (None = uniform)
    (3, 1, 1, None), (3, 5, 9, None), (7, 300, 200, None), (7, 600, 900, 400), (251, 450, 380, 200),
    (5, 1300, 700, None), (31, 200, 1100, 150), (2, 333, 250, None), (13, 800, 800, 640),
]


def dense(p, m, n, rank):
    if p == 2:
        return O.unpack_bits(synth.matrix(2, m, n, seed=21, rank=rank).numpy(), n)
    return synth.matrix(p, m, n, seed=21, rank=rank).numpy()


def rhs(A, p, k, seed):
    """k right-hand sides: images A x (consistent) with every third column
    moved off the column space by a left-kernel direction when one exists."""
    m, n = A.shape
    X0 = synth.uniform_u8(n, k, p, seed, 4).numpy().astype(np.int64)
    B = (A.astype(np.int64) @ X0) % p
    NL = O.nullspace_left(A, p)
    if NL.shape[0]:
        y = NL[0].astype(np.int64)
        e = np.zeros(m, np.int64)
        e[np.nonzero(y)[0][0]] = 1
        B[:, ::3] = (B[:, ::3] + e[:, None]) % p
    return B.astype(np.uint8)


@pytest.mark.parametrize("p,m,n,rank", CASES)
def test_nullspaces_u8(p, m, n, rank):
    A = dense(p, m, n, rank)
    res = gfe.echelon(torch.from_numpy(A).to(DEV), p)
    for side, ref in (("left", O.nullspace_left(A, p)), ("right", O.nullspace_right(A, p))):
        got = gfe.nullspace(res, p, m, n, side=side).cpu().numpy()
        assert got.shape == ref.shape, side
        assert np.array_equal(got, ref), (side, np.argwhere(got != ref)[:5])


@pytest.mark.parametrize("p,m,n,rank", CASES)
@pytest.mark.parametrize("k", [1, 70])
def test_solve_u8(p, m, n, rank, k):
    A = dense(p, m, n, rank)
    B = rhs(A, p, k, seed=m + k)
    res = gfe.echelon(torch.from_numpy(A).to(DEV), p)
    X, ok = gfe.solve(res, p, m, n, torch.from_numpy(B).to(DEV))
    Xr, okr = O.solve(A, p, B)
    assert np.array_equal(ok.cpu().numpy().astype(bool), okr)
    assert np.array_equal(X.cpu().numpy(), Xr)


@pytest.mark.parametrize("m,n,rank", [(1, 1, None), (200, 130, None), (700, 1100, 500), (1300, 900, None)])
def test_nullspaces_and_solve_gf2_bits(m, n, rank):
    Aw = synth.matrix(2, m, n, seed=23, rank=rank)
    A = O.unpack_bits(Aw.numpy(), n)
    res = gfe.echelon(Aw.to(DEV), 2, n=n)
    for side, ref, cols in (("left", O.nullspace_left(A, 2), m), ("right", O.nullspace_right(A, 2), n)):
        got = gfe.nullspace(res, 2, m, n, side=side)
        g = O.unpack_bits(got.cpu().numpy(), cols) if got.numel() else np.zeros((0, cols), np.uint8)
        assert np.array_equal(g, ref), side
    k = 130
    B = rhs(A, 2, k, seed=5)
    Bw = torch.from_numpy(O.pack_bits(B).view(np.int64)).to(DEV)
    X, ok = gfe.solve(res, 2, m, n, Bw, k=k)
    Xr, okr = O.solve(A, 2, B)
    assert np.array_equal(ok.cpu().numpy().astype(bool), okr)
    assert np.array_equal(O.unpack_bits(X.cpu().numpy(), k), Xr)


@pytest.mark.parametrize("p", [2, 7, 251])
def test_solve_and_nullspaces_edge_cases(p):
    for A in [np.zeros((6, 4), np.uint8), np.eye(5, dtype=np.uint8), np.zeros((0, 3), np.uint8),
              np.zeros((3, 0), np.uint8), np.tile(np.arange(4, dtype=np.uint8) % p, (5, 1))]:
        m, n = A.shape
        res = gfe.echelon(torch.from_numpy(A).to(DEV), p)
        for side, ref in (("left", O.nullspace_left(A, p)), ("right", O.nullspace_right(A, p))):
            got = gfe.nullspace(res, p, m, n, side=side).cpu().numpy()
            assert got.shape == ref.shape and np.array_equal(got, ref), (A.shape, side)
        B = synth.uniform_u8(m, 3, p, 9, 0).numpy()
        X, ok = gfe.solve(res, p, m, n, torch.from_numpy(B).to(DEV))
        Xr, okr = O.solve(A, p, B)
        assert np.array_equal(ok.cpu().numpy().astype(bool), okr), A.shape
        assert np.array_equal(X.cpu().numpy(), Xr), A.shape


def test_solve_after_batch_and_nonblocking_stream():
    """A batched result serves the same calls; solve on a side stream returns
    complete results."""
    p, m, n = 7, 900, 600
    A = dense(p, m, n, None)
    res = gfe.batch_echelon([(torch.from_numpy(A).to(DEV), p)])[0]
    B = rhs(A, p, 9, seed=3)
    side = torch.cuda.Stream()
    Bd = torch.from_numpy(B).to(DEV)
    torch.cuda.synchronize()
    X, ok = gfe.solve(res, p, m, n, Bd, stream=side)
    side.synchronize()
    Xr, okr = O.solve(A, p, B)
    assert np.array_equal(X.cpu().numpy(), Xr) and np.array_equal(ok.cpu().numpy().astype(bool), okr)
