"""The single-block echelonisation (job ECH) kernels on matrices that fit one
leaf, element by element against the oracle (GPU).

A matrix of at most 64 columns and at most 256 rows (p > 2), or at most 1024
rows for p <= 13, is one leaf launch.  The cases aim at the eight-column
groups of the leaves:
* group boundaries and ragged last groups;
* groups without a pivot, and groups whose columns only partly take one;
* rank 0 and full rank;
* rows that become zero;
* the 256-row cut between the fp32 leaf and the byte leaf for small p.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1806_04211_gb300 import gfe, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def compare(A, p):
    m, n = A.shape
    got = gfe.echelon(torch.from_numpy(np.ascontiguousarray(A)).to(DEV), p)
    ref = O.echelon(A, p)
    assert got["rank"] == ref["rank"], (m, n)
    for k in ("rho", "ups"):
        assert np.array_equal(got[k].cpu().numpy(), ref[k]), k
    for k in ("R", "M", "K"):
        g = got[k].cpu().numpy()
        assert g.shape == ref[k].shape, (k, g.shape, ref[k].shape)
        assert np.array_equal(g, ref[k]), (k, np.argwhere(g != ref[k])[:5])


def dense(p, m, n, seed, rank=None):
    return synth.matrix(p, m, n, seed=seed, rank=rank).numpy()


FIELDS = [3, 7, 13, 17, 31, 37, 193, 251]


@pytest.mark.parametrize("p", FIELDS)
@pytest.mark.parametrize("m,n", [(1, 1), (5, 3), (8, 8), (9, 9), (31, 64), (64, 7), (100, 57), (256, 64), (255, 63)])
def test_leaf_shapes(p, m, n):
    compare(dense(p, m, n, seed=m * 131 + n), p)


@pytest.mark.parametrize("p", FIELDS)
@pytest.mark.parametrize("rank", [0, 1, 7, 8, 9, 40])
def test_leaf_low_rank(p, rank):
    compare(dense(p, 200, 64, seed=rank + 5, rank=rank), p)


@pytest.mark.parametrize("p", FIELDS)
def test_leaf_groups_without_pivots(p):
    """Columns 8..15 are zero (a whole group takes no pivot), column 20 is a
    multiple of column 3 and 30..33 repeat 26..29 (groups that take fewer
    pivots than columns), and rows 10..19 repeat rows 0..9."""
    A = dense(p, 180, 64, seed=p)
    A[:, 8:16] = 0
    A[:, 20] = (A[:, 3].astype(np.int64) * 5 % p).astype(np.uint8)
    A[:, 30:34] = A[:, 26:30]
    A[10:20] = A[0:10]
    compare(A, p)


@pytest.mark.parametrize("p", [3, 5, 7, 11, 13])
@pytest.mark.parametrize("m,rank", [(1024, None), (700, None), (257, None), (1024, 30), (999, 64)])
def test_byte_leaf_rows(p, m, rank):
    """Beyond 256 rows the byte leaf takes p <= 13; at most 256 rows go to the
    fp32 leaf (257 is the first byte-leaf size)."""
    compare(dense(p, m, 64, seed=m + p, rank=rank), p)


@pytest.mark.parametrize("p", [17, 251])
def test_leaf_entries_at_the_bound(p):
    """Entries of p - 1: everywhere (rank 1), and in place of every zero of a
    random matrix, so the updates add the largest products."""
    compare(np.full((256, 64), p - 1, dtype=np.uint8), p)  # rank 1
    B = dense(p, 256, 64, seed=3)
    B[B == 0] = p - 1
    compare(B, p)
