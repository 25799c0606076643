"""The planner (Steps 1-3 of the Chief, the recursive ECH, the batch entry
point) run on the CPU against stand-ins of the CUDA runtime and CPU
restatements of the jobs (tests/plansim/sim.cpp): its results equal the
oracle's, every buffer access stays in bounds, and no access of one stream
is unordered with a conflicting access of another (the two-stream schedule
of Step 1 is ordered by events alone).  No GPU needed."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from conftest import ROOT
from oracle import oracle as O
from paper_1806_04211_gb300 import gfe

CSRC = os.path.join(ROOT, "paper_1806_04211_gb300", "csrc")
SIMDIR = os.path.join(ROOT, "tests", "plansim")
LIB = os.path.join(SIMDIR, "_build", "libgfe_plansim.so")


def cuda_include():
    for d in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


@pytest.fixture(scope="module")
def sim():
    inc = cuda_include()
    if shutil.which("g++") is None or inc is None:
        pytest.skip("g++ or the CUDA headers are not available")
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    srcs = [os.path.join(CSRC, "gfe_chief.cu"), os.path.join(CSRC, "gfe_api.cu")]
    cmd = ["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-Wl,-Bsymbolic", "-x", "c++"] + srcs + \
          ["-x", "none", os.path.join(SIMDIR, "sim.cpp"), "-I", inc, "-I", os.path.join(ROOT, "include"),
           "-I", CSRC, "-o", LIB, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    L = ctypes.CDLL(LIB)
    L.sim_register.argtypes = [ctypes.c_void_p, ctypes.c_size_t]
    L.sim_races.restype = ctypes.c_long
    for name, (res, args) in gfe.SIGNATURES.items():
        if hasattr(L, name):
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
    yield L
    L.gfe_set_block_policy(0, 0)


def races(L):
    n = L.sim_races()
    L.sim_race_reset()
    return n


def run(L, A, p, n=None, flags=1):
    bits = A.dtype != np.uint8
    m = A.shape[0]
    nn = n if bits else A.shape[1]
    mat = gfe.GfeMatrix(p, m, nn, 1 if bits else 0, A.ctypes.data, A.strides[0])
    mn = min(m, nn)

    def out(rows, cols):
        if bits:
            return np.zeros((max(rows, 1), gfe.words_per_row(max(cols, 1))), np.uint64)
        return np.zeros((max(rows, 1), max(cols, 1)), np.uint8)

    rank = np.zeros(1, np.int64)
    pc = np.zeros(max(mn, 1), np.int64)
    pr = np.zeros(max(mn, 1), np.int64)
    R, M, K = out(mn, nn), out(mn, mn), out(m, mn)
    for a in (A, rank, pc, pr, R, M, K):
        L.sim_register(a.ctypes.data, a.nbytes)
    res = gfe.GfeResult(rank.ctypes.data, pc.ctypes.data, pr.ctypes.data, R.ctypes.data, R.strides[0],
                        M.ctypes.data, M.strides[0], K.ctypes.data, K.strides[0], None, 0, None, 0)
    need = ctypes.c_size_t(0)
    assert L.gfe_query_workspace(ctypes.byref(mat), flags, ctypes.byref(need)) == 0
    ws = np.zeros(need.value, np.uint8)
    L.sim_register(ws.ctypes.data, ws.nbytes)
    st = L.gfe_echelon(ctypes.byref(mat), ctypes.byref(res), flags, ws.ctypes.data, ws.nbytes, None)
    assert st == 0, L.gfe_last_error()
    r = int(rank[0])
    d = dict(rank=r, rho=pr[:r], ups=pc[:r])
    if bits:
        d.update(R=R[:r] if r else R[:0], M=M[:r], K=K[:m - r])
    else:
        d.update(R=R[:r, :nn - r], M=M[:r, :r], K=K[:m - r, :r])
    return d


def check(L, A, p):
    got = run(L, A, p)
    ref = O.echelon(A, p)
    assert got["rank"] == ref["rank"]
    for k in ("rho", "ups", "R", "M", "K"):
        assert np.array_equal(got[k], ref[k]), k
    assert races(L) == 0


def check_gf2(L, A):
    m, n = A.shape
    W = O.pack_bits(A)
    got = run(L, W, 2, n=n)
    ref = O.echelon_gf2(W, m, n)
    r = ref["rank"]
    assert got["rank"] == r
    for k in ("rho", "ups"):
        assert np.array_equal(got[k], ref[k]), k
    for k, cols in (("R", n - r), ("M", r), ("K", r)):
        rows = ref[k].shape[0] if ref[k].size else 0
        if rows and cols:
            assert np.array_equal(O.unpack_bits(got[k], cols)[:rows], O.unpack_bits(ref[k], cols)), k
    assert races(L) == 0


# (threshold, block): a top-level Chief over small blocks; blocks wider than
# a leaf (128, 96 > 64 columns for p > 2) make the ECH of each block a Chief
# of its own, so two levels of side streams run at once
POLICIES = [(40, 16), (100, 48), (150, 128), (130, 96)]


@pytest.mark.parametrize("thr,blk", POLICIES)
def test_planner_matches_oracle_without_races(sim, thr, blk):
    assert sim.gfe_set_block_policy(thr, blk) == 0
    rng = np.random.RandomState(thr + blk)
    for trial in range(10):
        p = [3, 5, 7, 2, 13, 251, 31][trial % 7]
        m, n = rng.randint(1, 200), rng.randint(1, 200)
        kind = trial % 3
        if kind == 0:
            A = rng.randint(0, p, (m, n))
        elif kind == 1:
            k = rng.randint(0, min(m, n) + 1)
            A = (rng.randint(0, p, (m, k)) @ rng.randint(0, p, (k, n))) % p
        else:
            A = rng.randint(0, p, (m, n)) * (rng.rand(m, n) < 0.05)
        A = A.astype(np.uint8)
        if p == 2:
            check_gf2(sim, A)
        else:
            check(sim, A, p)
    sim.gfe_set_block_policy(0, 0)


def test_planner_sim_detects_a_planted_race(sim):
    """The checker itself: two copies on different streams with no event
    between them, writing the same bytes, must be reported."""
    buf = np.zeros(64, np.uint8)
    src = np.ones(64, np.uint8)
    sim.sim_register(buf.ctypes.data, buf.nbytes)
    sim.sim_register(src.ctypes.data, src.nbytes)
    s1, s2 = ctypes.c_void_p(), ctypes.c_void_p()
    sim.cudaStreamCreateWithFlags(ctypes.byref(s1), 1)
    sim.cudaStreamCreateWithFlags(ctypes.byref(s2), 1)
    cp = sim.cudaMemcpyAsync
    cp.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p]
    races(sim)
    cp(buf.ctypes.data, src.ctypes.data, 64, 3, s1)  # device to device
    cp(buf.ctypes.data, src.ctypes.data, 64, 3, s2)
    assert races(sim) > 0
    # ordered by an event: no race
    ev = ctypes.c_void_p()
    sim.cudaEventCreate(ctypes.byref(ev))
    cp(buf.ctypes.data, src.ctypes.data, 64, 3, s1)
    sim.cudaEventRecord(ev, s1)
    sim.cudaStreamWaitEvent(s2, ev, 0)
    cp(buf.ctypes.data, src.ctypes.data, 64, 3, s2)
    assert races(sim) == 0


@pytest.mark.parametrize("policy", [1, 2])
def test_batch_matches_oracle_without_races(sim, policy):
    """gfe_batch_echelon: two workers, each on its own stream with its own
    side streams and workspace slice, fenced to the caller's stream; the
    workers either poll (1) or wait on their own blocking event (2)."""
    assert sim.gfe_set_batch_workers(2) == 0
    assert sim.gfe_set_wait_policy(policy) == 0
    rng = np.random.RandomState(5)
    mats = [(rng.randint(0, p, (rng.randint(1, 150), rng.randint(1, 150))).astype(np.uint8), p)
            for p in [3, 5, 7, 251, 2, 3, 11, 13]]
    args, outs, keep = [], [], []
    for A, p in mats:
        m, n = A.shape
        sim.sim_register(A.ctypes.data, A.nbytes)
        mn = min(m, n)
        rank = np.zeros(1, np.int64)
        pc = np.zeros(max(mn, 1), np.int64)
        pr = np.zeros(max(mn, 1), np.int64)
        R = np.zeros((max(mn, 1), max(n, 1)), np.uint8)
        M = np.zeros((max(mn, 1), max(mn, 1)), np.uint8)
        K = np.zeros((max(m, 1), max(mn, 1)), np.uint8)
        for a in (rank, pc, pr, R, M, K):
            sim.sim_register(a.ctypes.data, a.nbytes)
        keep.append((rank, pc, pr, R, M, K))
        args.append(gfe.GfeMatrix(p, m, n, 0, A.ctypes.data, A.strides[0]))
        outs.append(gfe.GfeResult(rank.ctypes.data, pc.ctypes.data, pr.ctypes.data, R.ctypes.data, R.strides[0],
                                  M.ctypes.data, M.strides[0], K.ctypes.data, K.strides[0], None, 0, None, 0))
    arr = (gfe.GfeMatrix * len(args))(*args)
    res = (gfe.GfeResult * len(args))(*outs)
    need = ctypes.c_size_t(0)
    assert sim.gfe_query_batch_workspace(arr, len(args), 1, ctypes.byref(need)) == 0
    ws = np.zeros(need.value, np.uint8)
    sim.sim_register(ws.ctypes.data, ws.nbytes)
    assert sim.gfe_batch_echelon(arr, res, len(args), 1, ws.ctypes.data, ws.nbytes, None) == 0, sim.gfe_last_error()
    for (A, p), (rank, pc, pr, R, M, K) in zip(mats, keep):
        ref = O.echelon(A, p)
        r = ref["rank"]
        m, n = A.shape
        assert int(rank[0]) == r
        assert np.array_equal(pr[:r], ref["rho"]) and np.array_equal(pc[:r], ref["ups"])
        assert np.array_equal(M[:r, :r], ref["M"]) and np.array_equal(K[:m - r, :r], ref["K"])
        assert np.array_equal(R[:r, :n - r], ref["R"])
    assert races(sim) == 0
    sim.gfe_set_batch_workers(0)
    sim.gfe_set_wait_policy(0)


@pytest.mark.parametrize("p", [7, 251, 2])
def test_rank_deficient_wide_zero_blocks(sim, p):
    """Past the rank whole row blocks become zero; the planner tests such
    blocks (larger than a leaf) for zero before their ECH.  Results and
    ordering must not change."""
    assert sim.gfe_set_block_policy(150, 128) == 0
    rng = np.random.RandomState(p)
    m, n, k = 300, 700, 40
    A = ((rng.randint(0, p, (m, k)) @ rng.randint(0, p, (k, n))) % p).astype(np.uint8)
    if p == 2:
        check_gf2(sim, A)
    else:
        check(sim, A, p)
    sim.gfe_set_block_policy(0, 0)


def test_small_batch_two_formats_without_races(sim):
    """A batch of bit-packed GF(2) and byte matrices (small and large p) all
    taken by the one-launch small-matrix path, one stream per kind of
    kernel: oracle results, no unordered access."""
    rng = np.random.RandomState(11)
    specs = [(2, 70, 130), (3, 40, 33), (2, 1, 65), (13, 90, 64), (7, 17, 1), (2, 128, 128), (251, 30, 40)]
    keep, args, outs, refs = [], [], [], []
    for p, m, n in specs:
        mn = min(m, n)
        if p == 2:
            B = rng.randint(0, 2, (m, n)).astype(np.uint8)
            if m > 60:
                B[m // 2:] = 0  # rank-deficient
            A = O.pack_bits(B)
            ref = O.echelon_gf2(A, m, n)
            wr = lambda c: max(((c + 63) // 64 + 1) // 2 * 2, 2)  # the oracle's even word count
            R = np.zeros((max(mn, 1), wr(n)), np.uint64)
            M = np.zeros((max(mn, 1), wr(mn)), np.uint64)
            K = np.zeros((max(m, 1), wr(mn)), np.uint64)
            fmt = 1
        else:
            A = rng.randint(0, p, (m, n)).astype(np.uint8)
            ref = O.echelon(A, p)
            R = np.zeros((max(mn, 1), max(n, 1)), np.uint8)
            M = np.zeros((max(mn, 1), max(mn, 1)), np.uint8)
            K = np.zeros((max(m, 1), max(mn, 1)), np.uint8)
            fmt = 0
        rank = np.zeros(1, np.int64)
        pc = np.zeros(max(mn, 1), np.int64)
        pr = np.zeros(max(mn, 1), np.int64)
        for a in (A, rank, pc, pr, R, M, K):
            sim.sim_register(a.ctypes.data, a.nbytes)
        keep.append((A, rank, pc, pr, R, M, K))
        refs.append(ref)
        args.append(gfe.GfeMatrix(p, m, n, fmt, A.ctypes.data, A.strides[0]))
        outs.append(gfe.GfeResult(rank.ctypes.data, pc.ctypes.data, pr.ctypes.data, R.ctypes.data, R.strides[0],
                                  M.ctypes.data, M.strides[0], K.ctypes.data, K.strides[0], None, 0, None, 0))
    arr = (gfe.GfeMatrix * len(args))(*args)
    res = (gfe.GfeResult * len(args))(*outs)
    need = ctypes.c_size_t(0)
    assert sim.gfe_query_batch_workspace(arr, len(args), 1, ctypes.byref(need)) == 0
    ws = np.zeros(need.value, np.uint8)
    sim.sim_register(ws.ctypes.data, ws.nbytes)
    assert sim.gfe_batch_echelon(arr, res, len(args), 1, ws.ctypes.data, ws.nbytes, None) == 0, sim.gfe_last_error()
    for (p, m, n), ref, (A, rank, pc, pr, R, M, K) in zip(specs, refs, keep):
        r = ref["rank"]
        assert int(rank[0]) == r, (p, m, n)
        assert np.array_equal(pr[:r], ref["rho"]) and np.array_equal(pc[:r], ref["ups"])
        for got, want in ((R, ref["R"]), (M, ref["M"]), (K, ref["K"])):
            want = np.asarray(want)
            if want.size:
                assert np.array_equal(got[:want.shape[0], :want.shape[1]].view(want.dtype), want), (p, m, n)
    assert races(sim) == 0


def test_batch_split_by_side_and_work(sim):
    """The work cut-off and the side limit move matrices between the
    one-launch kernel and the workers: the workspace query follows the
    split (a small matrix needs m x ceil16(n) bytes, a worker its slice)."""
    def need(side, work):
        assert sim.gfe_set_batch_small_max(side, ctypes.c_double(work)) == 0
        A = np.zeros((300, 300), np.uint8)
        arr = (gfe.GfeMatrix * 1)(gfe.GfeMatrix(7, 300, 300, 0, A.ctypes.data, 300))
        n = ctypes.c_size_t(0)
        assert sim.gfe_query_batch_workspace(arr, 1, 1, ctypes.byref(n)) == 0
        return n.value
    small = need(2048, 0.0)
    assert small < 300 * 304 + 4096          # the matrix itself and the job table
    assert need(2048, 1e6) > small           # 300^3 > 1e6: a worker slice
    assert need(256, 0.0) > small            # side 300 > 256: a worker slice
    sim.gfe_set_batch_small_max(2048, ctypes.c_double(0.0))
