"""Pins for the CPU oracle: everything here is fixed by the paper or by the
mathematics, never by the oracle itself (CPU only)."""
import itertools
import math

import numpy as np
import pytest

from conftest import load_golden
from oracle import oracle as O
from paper_1806_04211_gb300 import synth

# ---------------------------------------------------------------------------
# independent helpers (no oracle code)
# ---------------------------------------------------------------------------


def rowspace(A, p):
    """All p^m combinations of the rows of A, as a set of byte strings."""
    m, n = A.shape
    if m == 0:
        return {bytes(n)}
    coeffs = np.array(list(itertools.product(range(p), repeat=m)), dtype=np.int64)
    vecs = (coeffs @ A.astype(np.int64)) % p
    return {v.astype(np.uint8).tobytes() for v in vecs}


def brute_rank(A, p):
    s = len(rowspace(A, p))
    r = round(math.log(s, p))
    assert p ** r == s
    return r


def check_neg_rref(E_top, ups, p):
    """E_top in the paper's negative reduced echelon form with pivots ups."""
    r, n = E_top.shape
    for l in range(r):
        row = E_top[l]
        nz = np.nonzero(row)[0]
        assert len(nz) and nz[0] == ups[l], "leading entry must be the pivot"
        assert row[ups[l]] == p - 1, "pivot entry is -1"
        for l2 in range(r):
            if l2 != l:
                assert E_top[l2, ups[l]] == 0, "pivot column cleared"
    assert all(ups[i] < ups[i + 1] for i in range(r - 1))


def assemble_E(res, m, n, p):
    r = res["rank"]
    E = np.zeros((m, n), np.uint8)
    non = [c for c in range(n) if c not in set(res["ups"].tolist())]
    for l in range(r):
        E[l, res["ups"][l]] = p - 1
        E[l, non] = res["R"][l]
    return E


def assemble_T(res, m, p):
    r = res["rank"]
    T = np.zeros((m, m), np.uint8)
    rho = res["rho"]
    non = [x for x in range(m) if x not in set(rho.tolist())]
    for l in range(r):
        T[l, rho] = res["M"][l]
    for t, x in enumerate(non):
        T[r + t, rho] = res["K"][t]
        T[r + t, x] = 1
    return T


def full_check(A, p, res):
    """T A = E, E in -RREF, rowspace(E_top) = rowspace(A), rho = row rank profile."""
    m, n = A.shape
    E = assemble_E(res, m, n, p)
    T = assemble_T(res, m, p)
    assert np.array_equal((T.astype(np.int64) @ A.astype(np.int64)) % p, E)
    r = res["rank"]
    check_neg_rref(E[:r], res["ups"], p)
    assert not E[r:].any()


# ---------------------------------------------------------------------------
# the paper's worked example (Section 2.2)
# ---------------------------------------------------------------------------

G = load_golden("paper_example_f3.txt")


def test_paper_example_top_left_ech():
    C = np.array(G["C"], np.uint8)
    H = C[:3, :3]
    res = O.echelon(H, 3, want_E=True, want_T=True)
    assert res["rank"] == 2
    assert res["rho"].tolist() == G["ECH_TL_rho"][0]
    assert res["ups"].tolist() == G["ECH_TL_gamma"][0]
    assert np.array_equal(res["M"], np.array(G["ECH_TL_M"], np.uint8))
    assert np.array_equal(res["K"], np.array(G["ECH_TL_K"], np.uint8))
    assert np.array_equal(res["R"], np.array(G["ECH_TL_R"], np.uint8))
    # the printed (M 0; K 1) P_rho H P_gamma
    P = np.array(G["ECH_TL_product"], np.int64)
    rho, ups = res["rho"], res["ups"]
    nonr = [x for x in range(3) if x not in rho]
    nonc = [c for c in range(3) if c not in ups]
    L = np.zeros((3, 3), np.int64)
    L[:2, :2] = res["M"]
    L[2:, :2] = res["K"]
    L[2, 2] = 1
    PH = H[list(rho) + nonr][:, list(ups) + nonc].astype(np.int64)
    assert np.array_equal((L @ PH) % 3, P)


def test_paper_example_updaterow_values():
    """UpdateRow steps (3) and (6) on the top-right block with the oracle's
    M, K, rho reproduce the printed M V and W + K V."""
    C = np.array(G["C"], np.uint8)
    res = O.echelon(C[:3, :3], 3)
    Z = C[:3, 3:].astype(np.int64)
    V = Z[res["rho"]]
    W = Z[[x for x in range(3) if x not in res["rho"]]]
    assert np.array_equal((res["M"].astype(np.int64) @ V) % 3, np.array(G["UR_MV"]))
    assert np.array_equal((W + res["K"].astype(np.int64) @ V) % 3, np.array(G["UR_W_plus_KV"]))
    # ClearDown on the bottom-left block and the bottom-right update
    BL = C[3:, :3].astype(np.int64)
    sel, non = BL[:, res["ups"]], BL[:, [2]]
    assert np.array_equal((non + sel @ res["R"].astype(np.int64)) % 3, np.array(G["CD_bottom_left"]))
    MV = (res["M"].astype(np.int64) @ V) % 3
    BR = (C[3:, 3:].astype(np.int64) + sel @ MV) % 3
    assert np.array_equal(BR, np.array(G["BR_after"]))


def test_paper_example_whole_matrix_row_equivalent():
    """The intermediate matrix printed at the end of the example is row-equivalent
    to C, so both have the same (unique) reduced echelon form and rank."""
    C = np.array(G["C"], np.uint8)
    C2 = np.array(G["C_after"], np.uint8)
    a = O.echelon(C, 3, want_E=True, want_T=True)
    b = O.echelon(C2, 3, want_E=True)
    assert a["rank"] == b["rank"] == brute_rank(C, 3)
    assert np.array_equal(a["E"], b["E"])
    assert np.array_equal(a["ups"], b["ups"])
    full_check(C, 3, a)
    assert rowspace(C, 3) == rowspace(C2, 3)


# ---------------------------------------------------------------------------
# brute force on every tiny matrix
# ---------------------------------------------------------------------------


def count_rank(p, m, n, r):
    """Number of m x n matrices of rank r over GF(p)."""
    num = 1
    for i in range(r):
        num *= (p ** m - p ** i) * (p ** n - p ** i)
    den = 1
    for i in range(r):
        den *= p ** r - p ** i
    return num // den


def greedy_rho(A, p):
    """Row x is a pivot row iff the rank grows when x is added (brute force)."""
    rho, prev = [], 0
    for x in range(A.shape[0]):
        rk = brute_rank(A[: x + 1], p)
        if rk > prev:
            rho.append(x)
        prev = rk
    return rho


@pytest.mark.parametrize("p,m,n", [(3, 3, 3), (3, 2, 4), (2, 3, 5), (2, 4, 3)])
def test_brute_force_all_matrices(p, m, n):
    hist = {}
    for flat in itertools.product(range(p), repeat=m * n):
        A = np.array(flat, np.uint8).reshape(m, n)
        res = O.echelon(A, p)
        r = res["rank"]
        hist[r] = hist.get(r, 0) + 1
        E = assemble_E(res, m, n, p)
        # rowspace(E_top) == rowspace(A): E_top = -RREF(A)
        assert rowspace(E[:r], p) == rowspace(A, p)
        check_neg_rref(E[:r], res["ups"], p)
        assert res["rho"].tolist() == greedy_rho(A, p)
        full_check(A, p, res)
    for r in range(min(m, n) + 1):
        assert hist.get(r, 0) == count_rank(p, m, n, r)
    assert sum(hist.values()) == p ** (m * n)


def test_brute_force_gf2_4x4_rank_histogram_packed():
    """Every 4 x 4 GF(2) matrix through the bit-packed oracle."""
    m = n = 4
    hist = {}
    for v in range(1 << 16):
        bits = np.array([(v >> k) & 1 for k in range(16)], np.uint8).reshape(4, 4)
        res = O.echelon_gf2(O.pack_bits(bits), m, n)
        hist[res["rank"]] = hist.get(res["rank"], 0) + 1
        if v % 97 == 0:
            assert res["rank"] == brute_rank(bits, 2)
    for r in range(5):
        assert hist.get(r, 0) == count_rank(2, 4, 4, r)


# ---------------------------------------------------------------------------
# closed forms and special cases
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("p", [2, 3, 7, 251])
def test_zero_matrix(p):
    A = np.zeros((5, 7), np.uint8)
    res = O.echelon(A, p, want_E=True, want_T=True)
    assert res["rank"] == 0 and not res["E"].any()
    assert np.array_equal(res["T"], np.eye(5, dtype=np.uint8))


@pytest.mark.parametrize("p", [2, 3, 7, 251])
def test_identity(p):
    A = np.eye(6, dtype=np.uint8)
    res = O.echelon(A, p)
    assert res["rank"] == 6
    assert np.array_equal(res["M"], ((p - 1) * np.eye(6)).astype(np.uint8))
    assert res["rho"].tolist() == list(range(6)) == res["ups"].tolist()


def mat_inv_mod(A, p):
    """Inverse by Gauss-Jordan on (A | I) in plain Python (independent)."""
    n = A.shape[0]
    Mx = [[int(A[i][j]) for j in range(n)] + [int(i == j) for j in range(n)] for i in range(n)]
    for c in range(n):
        piv = next(i for i in range(c, n) if Mx[i][c] % p)
        Mx[c], Mx[piv] = Mx[piv], Mx[c]
        inv = pow(Mx[c][c], p - 2, p)
        Mx[c] = [(v * inv) % p for v in Mx[c]]
        for i in range(n):
            if i != c and Mx[i][c]:
                f = Mx[i][c]
                Mx[i] = [(a - f * b) % p for a, b in zip(Mx[i], Mx[c])]
    return np.array([row[n:] for row in Mx], np.int64)


@pytest.mark.parametrize("p", [3, 5, 7, 251])
def test_invertible_gives_minus_inverse(p):
    rng = np.random.RandomState(p)
    for _ in range(5):
        while True:
            A = rng.randint(0, p, (7, 7)).astype(np.uint8)
            if brute_rank(A[:, :], p) == 7 if p < 5 else True:
                try:
                    Ainv = mat_inv_mod(A, p)
                    break
                except StopIteration:
                    continue
        res = O.echelon(A, p, want_E=True, want_T=True)
        assert res["rank"] == 7
        assert np.array_equal(res["E"], ((p - 1) * np.eye(7)).astype(np.uint8))
        assert np.array_equal(res["T"].astype(np.int64), (-Ainv) % p)
        assert np.array_equal((A.astype(np.int64) @ res["T"]) % p, (-np.eye(7, dtype=np.int64)) % p)


@pytest.mark.parametrize("p", [2, 3, 251])
def test_permutation_matrix(p):
    perm = [3, 0, 4, 1, 2]
    A = np.zeros((5, 5), np.uint8)
    for i, j in enumerate(perm):
        A[i, j] = 1
    res = O.echelon(A, p, want_T=True)
    assert res["rank"] == 5
    # row l of M is -(row of A with its 1 in column l), as a coefficient vector on rows
    for l in range(5):
        src = perm.index(l)
        expect = np.zeros(5, np.uint8)
        expect[src] = p - 1
        assert np.array_equal(res["M"][l], expect)


@pytest.mark.parametrize("p", [2, 3, 7, 251])
def test_low_rank_product_exact_rank(p):
    """A = U V with U = [I; X], V = [I | Y] has rank exactly k; rho = first k
    rows, ups = first k columns, R = -Y (the -RREF of [I | Y])."""
    rng = np.random.RandomState(11)
    m, n, k = 9, 11, 4
    U = np.vstack([np.eye(k, dtype=np.int64), rng.randint(0, p, (m - k, k))])
    V = np.hstack([np.eye(k, dtype=np.int64), rng.randint(0, p, (k, n - k))])
    A = ((U @ V) % p).astype(np.uint8)
    res = O.echelon(A, p)
    assert res["rank"] == k
    assert res["rho"].tolist() == list(range(k)) and res["ups"].tolist() == list(range(k))
    assert np.array_equal(res["R"].astype(np.int64), (-V[:, k:]) % p)
    # K rows: row x = X_x . (first k rows) so K = -X (coefficients that cancel it)
    assert np.array_equal(res["K"].astype(np.int64), (-U[k:]) % p)


@pytest.mark.parametrize("p", [2, 3, 5])
def test_duplicate_row_k_is_minus_unit(p):
    rng = np.random.RandomState(3)
    A = rng.randint(0, p, (6, 8)).astype(np.uint8)
    A[4] = A[1]
    res = O.echelon(A, p)
    rho = res["rho"].tolist()
    assert 1 in rho and 4 not in rho
    non = [x for x in range(6) if x not in rho]
    krow = res["K"][non.index(4)]
    expect = np.zeros(len(rho), np.uint8)
    expect[rho.index(1)] = p - 1
    assert np.array_equal(krow, expect)


@pytest.mark.parametrize("p", [2, 3, 7, 251])
def test_random_full_check(p):
    rng = np.random.RandomState(5 + p)
    for (m, n) in [(1, 1), (1, 9), (9, 1), (13, 8), (8, 13), (30, 30)]:
        A = rng.randint(0, p, (m, n)).astype(np.uint8)
        res = O.echelon(A, p)
        full_check(A, p, res)
        # closed form M = -A[rho,ups]^{-1} checked through M A[rho,ups] = -I
        H = A[np.ix_(res["rho"], res["ups"])].astype(np.int64)
        assert np.array_equal((res["M"].astype(np.int64) @ H) % p, (-np.eye(res["rank"], dtype=np.int64)) % p)
        # K = A[rho_bar, ups] M
        non = [x for x in range(m) if x not in set(res["rho"].tolist())]
        Kc = (A[np.ix_(non, res["ups"])].astype(np.int64) @ res["M"].astype(np.int64)) % p
        assert np.array_equal(Kc, res["K"])


def test_empty_shapes():
    for (m, n) in [(0, 0), (0, 5), (5, 0)]:
        res = O.echelon(np.zeros((m, n), np.uint8), 3)
        assert res["rank"] == 0


def test_rejects_bad_p():
    with pytest.raises(ValueError):
        O.echelon(np.zeros((2, 2), np.uint8), 4)
    with pytest.raises(ValueError):
        O.echelon(np.zeros((2, 2), np.uint8), 257)


# ---------------------------------------------------------------------------
# bit-packed GF(2) oracle against brute force / the uint8 oracle's pins
# ---------------------------------------------------------------------------


def test_gf2_packed_matches_definition_random():
    rng = np.random.RandomState(7)
    for (m, n) in [(1, 1), (3, 70), (70, 3), (65, 129), (130, 64), (100, 100)]:
        bits = rng.randint(0, 2, (m, n)).astype(np.uint8)
        res = O.echelon_gf2(O.pack_bits(bits), m, n, want_E=True, want_T=True)
        r = res["rank"]
        unp = dict(rank=r, rho=res["rho"], ups=res["ups"],
                   M=O.unpack_bits(res["M"], r) if r else np.zeros((0, 0), np.uint8),
                   K=O.unpack_bits(res["K"], r) if m - r and r else np.zeros((m - r, r), np.uint8),
                   R=O.unpack_bits(res["R"], n - r) if r and n - r else np.zeros((r, n - r), np.uint8))
        full_check(bits, 2, unp)
        assert np.array_equal(O.unpack_bits(res["E"], n), assemble_E(unp, m, n, 2))
        assert np.array_equal(O.unpack_bits(res["T"], m), assemble_T(unp, m, 2))
        assert res["rho"].tolist() == greedy_rho(bits, 2) if m <= 8 else True


def test_full_rank_fraction_statistics():
    """Fraction of uniform random square matrices of full rank tends to
    prod_{i>=1} (1 - p^-i): 0.2888 for GF(2), 0.5601 for GF(3)."""
    rng = np.random.RandomState(1)
    for p, limit in [(2, 0.288788), (3, 0.560126)]:
        N, full = 3000, 0
        for _ in range(N):
            A = rng.randint(0, p, (12, 12)).astype(np.uint8)
            full += O.echelon(A, p)["rank"] == 12
        exact = np.prod([1 - p ** -i for i in range(1, 13)])
        assert abs(exact - limit) < 1e-3
        sigma = math.sqrt(exact * (1 - exact) / N)
        assert abs(full / N - exact) < 5 * sigma


# ---------------------------------------------------------------------------
# the certificate: accepts correct results, rejects planted mistakes
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("p", [3, 7, 251])
def test_certificate_accepts_and_rejects(p):
    rng = np.random.RandomState(p)
    A = rng.randint(0, p, (40, 50)).astype(np.uint8)
    A[30] = A[3]
    A[:, 7] = A[:, 2]
    res = O.echelon(A, p)
    assert O.certify(A, p, res) == 0
    for key in ("M", "K", "R"):
        bad = {k: (v.copy() if hasattr(v, "copy") else v) for k, v in res.items()}
        arr = bad[key]
        if arr.size == 0:
            continue
        i, j = rng.randint(0, arr.shape[0]), rng.randint(0, arr.shape[1])
        arr[i, j] = (arr[i, j] + 1) % p
        assert O.certify(A, p, bad) != 0, key
    bad = dict(res)
    rho = res["rho"].copy()
    rho[-1] = [x for x in range(40) if x not in rho][-1]
    bad["rho"] = np.sort(rho)
    assert O.certify(A, p, bad) != 0


def test_certificate_gf2_accepts_and_rejects():
    rng = np.random.RandomState(2)
    m, n = 90, 130
    bits = rng.randint(0, 2, (m, n)).astype(np.uint8)
    bits[50] = bits[10] ^ bits[20]
    W = O.pack_bits(bits)
    res = O.echelon_gf2(W, m, n)
    assert O.certify_gf2(W, m, n, res) == 0
    for key in ("M", "K", "R"):
        bad = dict(res)
        arr = res[key].copy()
        arr.view(np.uint64)[0, 0] ^= np.uint64(1 << 3)
        bad[key] = arr
        assert O.certify_gf2(W, m, n, bad) != 0, key


@pytest.mark.parametrize("m,n,rank", [(1, 1, None), (70, 130, None), (130, 70, None), (300, 300, 150),
                                      (257, 513, None), (600, 400, 250)])
def test_openmp_baseline_equals_oracle(m, n, rank):
    """The OpenMP timing baseline runs the oracle's GF(2) algorithm on all
    host cores; its outputs equal the oracle's."""
    A = synth.matrix(2, m, n, seed=77, rank=rank).numpy()
    ref = O.echelon_gf2(A, m, n)
    got = O.echelon_gf2_omp(A, m, n)
    assert got["rank"] == ref["rank"]
    for k in ("rho", "ups", "M", "K", "R"):
        assert np.array_equal(got[k], ref[k]), k


# ---------------------------------------------------------------------------
# solving and kernels (the paper's variant list, Section 1; Eq. (echelon))
# ---------------------------------------------------------------------------

def _all_vectors(p, length):
    return np.array(list(itertools.product(range(p), repeat=length)), dtype=np.int64).reshape(-1, length)


@pytest.mark.parametrize("p,m,n", [(3, 3, 3), (3, 2, 4), (2, 4, 3), (2, 3, 5)])
def test_nullspaces_brute_force(p, m, n):
    """Every matrix of the shape: the basis rows span exactly the vectors
    brute force finds in the left / right kernel, have the stated size, and
    are the identity on rho_bar / Ups_bar."""
    ys, xs = _all_vectors(p, m), _all_vectors(p, n)
    for flat in itertools.product(range(p), repeat=m * n):
        A = np.array(flat, dtype=np.uint8).reshape(m, n)
        A64 = A.astype(np.int64)
        left = {y.astype(np.uint8).tobytes() for y in ys if not ((y @ A64) % p).any()}
        right = {x.astype(np.uint8).tobytes() for x in xs if not ((A64 @ x) % p).any()}
        NL, NR = O.nullspace_left(A, p), O.nullspace_right(A, p)
        r = brute_rank(A, p)
        assert NL.shape == (m - r, m) and NR.shape == (n - r, n)
        assert rowspace(NL, p) == left
        assert rowspace(NR, p) == right


def test_nullspace_structure_random():
    for p, m, n, k in [(7, 40, 30, 12), (251, 25, 60, 20), (2, 50, 70, 33), (5, 60, 60, None)]:
        A = synth.matrix(p, m, n, seed=3, rank=k).numpy() if p != 2 else \
            O.unpack_bits(synth.matrix(2, m, n, seed=3, rank=k).numpy(), n)
        res = O.echelon(A, p)
        r = res["rank"]
        NL, NR = O.nullspace_left(A, p), O.nullspace_right(A, p)
        assert not ((NL.astype(np.int64) @ A) % p).any()
        assert not ((A.astype(np.int64) @ NR.T.astype(np.int64)) % p).any()
        nbar = np.setdiff1d(np.arange(m), res["rho"])
        ubar = np.setdiff1d(np.arange(n), res["ups"])
        assert np.array_equal(NL[:, nbar], np.eye(m - r, dtype=np.uint8))
        assert np.array_equal(NR[:, ubar], np.eye(n - r, dtype=np.uint8))


@pytest.mark.parametrize("p,m,n", [(3, 2, 3), (3, 3, 2), (2, 3, 3), (2, 2, 4)])
def test_solve_brute_force(p, m, n):
    """Every matrix and every right-hand side: consistent iff some x solves
    it (brute force); then the returned x solves it and is zero on the
    non-pivot columns, which brute force shows is unique."""
    xs, bs = _all_vectors(p, n), _all_vectors(p, m)
    for flat in itertools.product(range(p), repeat=m * n):
        A = np.array(flat, dtype=np.uint8).reshape(m, n)
        A64 = A.astype(np.int64)
        images = {}
        for x in xs:
            images.setdefault(((A64 @ x) % p).astype(np.uint8).tobytes(), []).append(x)
        X, ok = O.solve(A, p, bs.T.astype(np.uint8))
        ups = O.echelon(A, p)["ups"]
        ubar = np.setdiff1d(np.arange(n), ups)
        for j, b in enumerate(bs):
            sols = images.get(b.astype(np.uint8).tobytes(), [])
            assert ok[j] == bool(sols)
            if sols:
                assert np.array_equal((A64 @ X[:, j]) % p, b)
                zero_free = [x for x in sols if not x[ubar].any()]
                assert len(zero_free) == 1 and np.array_equal(zero_free[0], X[:, j])


def test_solve_random_consistent_and_planted():
    for p, m, n, k in [(7, 60, 45, 30), (251, 40, 70, 25), (2, 64, 64, 40), (3, 30, 80, None)]:
        A = (synth.matrix(p, m, n, seed=8, rank=k).numpy() if p != 2 else
             O.unpack_bits(synth.matrix(2, m, n, seed=8, rank=k).numpy(), n)).astype(np.uint8)
        X0 = synth.uniform_u8(n, 9, p, 8, 3).numpy().astype(np.int64)
        B = ((A.astype(np.int64) @ X0) % p).astype(np.uint8)
        r = O.echelon(A, p)["rank"]
        if r < m:  # a column outside the column space: a left-kernel vector y has y b != 0
            y = O.nullspace_left(A, p)[0].astype(np.int64)
            e = np.zeros(m, np.int64)
            e[np.nonzero(y)[0][0]] = 1
            B[:, 4] = (B[:, 4].astype(np.int64) + e) % p
        X, ok = O.solve(A, p, B)
        for j in range(B.shape[1]):
            if ok[j]:
                assert np.array_equal((A.astype(np.int64) @ X[:, j]) % p, B[:, j])
        assert ok.sum() == B.shape[1] - (1 if r < m else 0)
        if r < m:
            assert not ok[4]
