"""The batched form: independent matrices of mixed sizes and fields on
concurrent workers give exactly the single-call results (GPU)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1806_04211_gb300 import gfe, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def mixed(seed=0):
    rng = np.random.RandomState(seed)
    out = []
    for i in range(14):
        p = [2, 3, 5, 7, 251][i % 5]
        m, n = int(rng.randint(1, 700)), int(rng.randint(1, 700))
        rank = int(0.6 * min(m, n)) if i % 2 else None
        A = synth.matrix(p, m, n, seed=100 + i, rank=rank if rank else None)
        out.append((p, m, n, A))
    return out


@pytest.mark.parametrize("workers,policy", [(1, "spin"), (3, "auto"), (8, "spin"), (14, "block"), (40, "auto")])
def test_batch_matches_oracle_and_single_calls(workers, policy):
    """Polling and sleeping workers, fewer and more workers than matrices."""
    mats = mixed()
    args = [(A.to(DEV), p, n) if p == 2 else (A.to(DEV), p) for p, m, n, A in mats]
    gfe.set_wait_policy(policy)
    try:
        got = gfe.batch_echelon(args, workers=workers)
    finally:
        gfe.lib().gfe_set_batch_workers(0)
        gfe.set_wait_policy("auto")
    for (p, m, n, A), g, a in zip(mats, got, args):
        single = gfe.echelon(*a) if p != 2 else gfe.echelon(a[0], 2, n=n)
        assert g["rank"] == single["rank"]
        for k in ("rho", "ups", "R", "M", "K"):
            assert torch.equal(g[k], single[k]), (p, m, n, k)
        if p == 2:
            ref = O.echelon_gf2(A.numpy(), m, n)
        else:
            ref = O.echelon(A.numpy(), p)
        assert g["rank"] == ref["rank"]
        assert np.array_equal(g["rho"].cpu().numpy(), ref["rho"])
        if p != 2:
            assert np.array_equal(g["M"].cpu().numpy(), ref["M"])
            assert np.array_equal(g["K"].cpu().numpy(), ref["K"])
            assert np.array_equal(g["R"].cpu().numpy(), ref["R"])


def test_batch_empty_and_stream_order():
    assert gfe.batch_echelon([]) == []
    s = torch.cuda.Stream()
    A = synth.matrix(3, 300, 280, seed=4).to(DEV)
    with torch.cuda.stream(s):
        B = (A.to(torch.int32) * 2 % 3).to(torch.uint8)   # produced on s before the call
        got = gfe.batch_echelon([(B, 3)], stream=s)[0]
    ref = O.echelon(((A.cpu().numpy().astype(np.int32) * 2) % 3).astype(np.uint8), 3)
    assert got["rank"] == ref["rank"]
    assert np.array_equal(got["R"].cpu().numpy(), ref["R"])


def _check_vs_oracle(p, m, n, A, g):
    """Every output of one batch result against the oracle, bit-exact."""
    if p == 2:
        ref = O.echelon_gf2(A.numpy(), m, n)
    else:
        ref = O.echelon(A.numpy(), p)
    assert g["rank"] == ref["rank"], (p, m, n)
    assert np.array_equal(g["rho"].cpu().numpy(), ref["rho"]), (p, m, n)
    assert np.array_equal(g["ups"].cpu().numpy(), ref["ups"]), (p, m, n)
    for k in ("R", "M", "K"):
        got = g[k].cpu().numpy()
        want = np.asarray(ref[k])
        if p == 2:
            got, want = got.view(np.uint64), want.view(np.uint64)
        if got.size == 0 and want.size == 0:
            continue
        assert got.shape == want.shape and np.array_equal(got, want), (p, m, n, k)


# edge shapes of the one-launch small-matrix kernels: single rows / columns,
# ragged widths around the 16-byte vectors and 64-bit words, zero and
# rank-deficient inputs, fields of all three kernels (p = 11, 13: lazy
# reduction every 2 and every pivot step; p >= 17: the wide kernel), both
# sides of the 2048 limit
SMALL_CASES = [
    (3, 1, 1, None), (5, 1, 37, None), (7, 53, 1, None), (3, 17, 15, 0), (13, 64, 64, None),
    (11, 200, 129, 77), (13, 129, 200, None), (7, 300, 300, 180), (5, 511, 17, None), (3, 16, 2048, None),
    (2, 1, 1, None), (2, 1, 200, None), (2, 130, 1, None), (2, 65, 63, 0), (2, 257, 191, 100),
    (2, 700, 1500, None), (2, 2048, 64, None), (7, 2048, 40, 30),
    # 17 <= p <= 251: the panel in 16-bit lanes, the rest update in 32-bit lanes
    (17, 33, 47, None), (251, 300, 129, 77), (31, 129, 300, None), (101, 1, 40, None), (251, 64, 1, None),
    (193, 700, 700, 300), (251, 2048, 50, None), (37, 17, 15, 0), (251, 511, 511, None),
]


def test_small_kernel_edge_cases_match_oracle():
    mats = []
    for i, (p, m, n, rk) in enumerate(SMALL_CASES):
        A = synth.matrix(p, m, n, seed=900 + i, rank=rk if rk else None)
        mats.append((p, m, n, A.zero_() if rk == 0 else A))  # rank 0: the zero matrix
    args = [(A.to(DEV), p, n) for p, m, n, A in mats]
    gfe.set_batch_small_max(2048)
    got = gfe.batch_echelon(args)
    for (p, m, n, A), g in zip(mats, got):
        _check_vs_oracle(p, m, n, A, g)


def test_small_kernel_equals_worker_path_at_full_side():
    """2048 x 2048 (full rank and rank-deficient) by the one-launch kernel and
    by the blocked Chief on the workers: identical results; certified."""
    specs = [(2, 2048, 2048, None), (2, 2048, 2048, 1500), (7, 2048, 2048, None), (3, 1999, 2048, 1200),
             (13, 2048, 1500, None), (251, 2048, 2048, None), (17, 1800, 2048, 1100)]
    mats = [(p, m, n, synth.matrix(p, m, n, seed=950 + i, rank=rk)) for i, (p, m, n, rk) in enumerate(specs)]
    args = [(A.to(DEV), p, n) for p, m, n, A in mats]
    gfe.set_batch_small_max(2048, 1e12)  # above the default work cut-off: force the one-launch kernel
    small = gfe.batch_echelon(args)
    gfe.set_batch_small_max(0)
    try:
        chief = gfe.batch_echelon(args, workers=3)
    finally:
        gfe.set_batch_small_max(2048)
        gfe.lib().gfe_set_batch_workers(0)
    for (p, m, n, A), a, b in zip(mats, small, chief):
        assert a["rank"] == b["rank"], (p, m, n)
        for k in ("rho", "ups", "R", "M", "K"):
            assert torch.equal(a[k], b[k]), (p, m, n, k)
        res = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in a.items()}
        if p == 2:
            assert O.certify_gf2(A.numpy(), m, n, res) == 0
        else:
            assert O.certify(A.numpy(), p, res) == 0


def test_small_kernel_without_transform_and_null_outputs():
    """transform=False: M and K are not written; rank and pivots still are."""
    p, m, n = 5, 300, 250
    A = synth.matrix(p, m, n, seed=77, rank=140)
    got = gfe.batch_echelon([(A.to(DEV), p)], transform=False)[0]
    ref = O.echelon(A.numpy(), p)
    assert got["rank"] == ref["rank"] == 140
    assert np.array_equal(got["R"].cpu().numpy(), ref["R"])
    assert "M" not in got
