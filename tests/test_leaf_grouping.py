"""The grouped elimination of the leaf kernels, restated in numpy and checked
against the oracle (CPU).

The leaf kernels for p > 2 take eight columns at a time:
* a finder eliminates on the group's columns alone and records, for every
  row y, the multiple G[y][s] of the group's new pivot row s added to it;
* NP[s] is pivot row s as a combination of the rows Q_0 .. Q_s, Q_s being
  pivot row x_s as it stood at the group start plus the identity of its slot;
* row y becomes [y is no pivot of the group] * y + sum_s (G[y] NP)[s] Q_s.

The result must be the column-by-column Gauss-Jordan of the oracle, with the
same pivot rule (the topmost non-pivot row).  Here that identity is checked
on brute force, on random and low-rank inputs for every field, and through
the same read-out of rank, pivots, R, M and K that the kernels make, so a
mistake in the algebra the kernels rely on fails here, without a GPU.  The
arithmetic is exact integers reduced mod p; the kernels' value bounds (rows
below 64 p^2 + p, so below 2^24) are asserted on the way.
"""
import itertools

import numpy as np
import pytest

from oracle import oracle as O


def inverse(x, p):
    return pow(int(x), p - 2, p)


def grouped_leaf(H, p, G=8, drop_np_terms=False):
    """Rank, pivot rows, pivot columns, R, M, K of H (alpha x beta) by the
    grouped elimination, as residues.  drop_np_terms plants a mistake: NP[s]
    forgets the multiples the pivot row received earlier in its group."""
    a, b = H.shape
    h = H.astype(np.int64) % p
    t = np.zeros((a, b), np.int64)  # slot coefficients (slot s = the s-th pivot)
    piv = np.zeros(a, bool)
    slot_row, slot_col = [], []
    for c0 in range(0, b, G):
        kk = min(G, b - c0)
        pan = h[:, c0:c0 + kk] % p
        Gm = np.zeros((a, G), np.int64)
        NP = np.zeros((G, G), np.int64)
        xs = []
        cand = ~piv
        for k in range(kk):
            v = pan[:, k] % p
            rows = np.nonzero(cand & (v != 0))[0]
            if len(rows) == 0:
                continue
            x, s = int(rows[0]), len(xs)
            sc = (p - inverse(v[x], p)) % p  # makes the pivot -1
            newp = sc * (pan[x] % p) % p
            cmx = Gm[x, :s] @ NP[:s] % p if s and not drop_np_terms else np.zeros(G, np.int64)
            cmx[s] += 1
            NP[s] = sc * cmx % p
            others = np.arange(a) != x
            Gm[others, s] = v[others]
            pan[others] += v[others, None] * newp[None, :]
            assert pan.max() < 8 * p * p + p
            pan[x] = newp
            Gm[x] = 0
            Gm[x, s] = 1
            cand[x] = False
            xs.append(x)
            slot_row.append(x)
            slot_col.append(c0 + k)
        if not xs:
            continue
        ns = len(slot_row) - len(xs)
        Q = np.concatenate([h[xs] % p, t[xs] % p], axis=1)
        for s in range(len(xs)):
            Q[s, b + ns + s] += 1
        CM = Gm[:, :len(xs)] @ NP[:len(xs), :len(xs)] % p
        keep = np.ones(a, np.int64)
        keep[xs] = 0
        rows = keep[:, None] * np.concatenate([h, t], axis=1) + CM @ Q
        assert rows.max() < 64 * p * p + p < 2 ** 24
        h, t = rows[:, :b], rows[:, b:]
        piv[xs] = True
    h, t = h % p, t % p
    r = len(slot_row)
    rho = np.array(sorted(slot_row), dtype=np.int64)
    order = np.argsort(slot_col)  # the slots are the pivot columns in ascending order already
    assert np.array_equal(order, np.arange(r))
    ups = np.array(slot_col, dtype=np.int64)
    sorted_slot = [slot_row.index(y) for y in rho]  # slot of the l-th pivot row in row order
    non = [c for c in range(b) if c not in slot_col]
    M = np.array([[t[slot_row[l], sorted_slot[s]] for s in range(r)] for l in range(r)], np.int64).reshape(r, r)
    R = np.array([[h[slot_row[l], c] for c in non] for l in range(r)], np.int64).reshape(r, len(non))
    others = [y for y in range(a) if not piv[y]]
    K = np.array([[t[y, sorted_slot[s]] for s in range(r)] for y in others], np.int64).reshape(len(others), r)
    return dict(rank=r, rho=rho, ups=ups, R=R, M=M, K=K)


def check(A, p):
    check_with(A, p)


def check_with(A, p, **kw):
    got = grouped_leaf(A, p, **kw)
    ref = O.echelon(np.ascontiguousarray(A, dtype=np.uint8), p)
    assert got["rank"] == ref["rank"]
    for k in ("rho", "ups", "R", "M", "K"):
        assert np.array_equal(np.asarray(got[k], np.int64), np.asarray(ref[k], np.int64)), k


@pytest.mark.parametrize("p,m,n", [(3, 3, 3), (3, 2, 4), (5, 2, 3)])
def test_grouped_leaf_brute_force(p, m, n):
    """Every matrix of the shape (3^9, 3^8, 5^6 of them)."""
    for vals in itertools.product(range(p), repeat=m * n):
        check(np.array(vals, dtype=np.uint8).reshape(m, n), p)


def test_grouped_leaf_two_groups():
    """Seeded 3 x 11 and 11 x 3 matrices over F_3 (two groups, the second
    ragged) with their entries drawn from {0, 1, 2}."""
    rng = np.random.RandomState(11)
    for _ in range(1500):
        check(rng.randint(0, 3, (3, 11)).astype(np.uint8), 3)
        check(rng.randint(0, 3, (11, 3)).astype(np.uint8), 3)


FIELDS = [3, 5, 7, 11, 13, 17, 31, 37, 193, 251]


@pytest.mark.parametrize("p", FIELDS)
def test_grouped_leaf_random(p):
    rng = np.random.RandomState(p)
    for m, n, rank in [(60, 64, None), (64, 60, None), (40, 64, 20), (70, 33, 9), (17, 64, 0), (90, 64, 64)]:
        if rank is None:
            A = rng.randint(0, p, (m, n))
        else:
            A = rng.randint(0, p, (m, rank)) @ rng.randint(0, p, (rank, n)) % p
        A = A.astype(np.uint8)
        A[:, 8:16] = 0  # a group without pivots
        check(A, p)


@pytest.mark.parametrize("p", [7, 251])
def test_grouped_leaf_planted_mistake_is_caught(p):
    """Without the NP recursion (the pivot row's earlier multiples in its
    group) the result differs from the oracle: these checks would see it."""
    rng = np.random.RandomState(1)
    A = rng.randint(0, p, (40, 24)).astype(np.uint8)
    check(A, p)
    with pytest.raises(AssertionError):
        check_with(A, p, drop_np_terms=True)
