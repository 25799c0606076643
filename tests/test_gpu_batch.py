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


@pytest.mark.parametrize("workers", [1, 3, 8])
def test_batch_matches_oracle_and_single_calls(workers):
    mats = mixed()
    args = [(A.to(DEV), p, n) if p == 2 else (A.to(DEV), p) for p, m, n, A in mats]
    got = gfe.batch_echelon(args, workers=workers)
    gfe.lib().gfe_set_batch_workers(0)
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
