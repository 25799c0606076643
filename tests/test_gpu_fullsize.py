"""Full-size configurations (C2 n = 32768 bit-packed GF(2), C3 32768^2 GF(7)
and 20000 x 50000 GF(251) twin) in the launch configuration the benchmark
uses, checked by the oracle's certificate (exact structure checks plus
Freivalds' check of T A = E; the oracle itself is too slow at these sizes)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1806_04211_gb300 import gfe, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def host(d):
    return {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in d.items()}


@pytest.mark.parametrize("rank", [None, 24576])
def test_c2_gf2_32768_certificate(rank):
    n = 32768
    A = synth.matrix(2, n, n, seed=1, rank=rank, device=DEV)
    got = gfe.batch_echelon([(A, 2, n)], workers=1)[0]
    if rank is not None:
        assert got["rank"] == rank
    else:
        assert got["rank"] >= n - 8
    res = host(got)
    for k in ("M", "K", "R"):
        res[k] = np.ascontiguousarray(res[k]).view(np.uint64)
    assert O.certify_gf2(A.cpu().numpy(), n, n, res, seed=7) == 0


def test_c3_gf7_32768_certificate():
    n = 32768
    A = synth.matrix(7, n, n, seed=2, device=DEV)
    got = gfe.echelon(A, 7)
    assert got["rank"] >= n - 4
    assert O.certify(A.cpu().numpy(), 7, host(got), nvec=4, seed=3) == 0


def test_c3_gf251_rect_twin_certificate():
    m, n = 20000, 50000
    A = synth.matrix(251, m, n, seed=3, rank=12000, device=DEV)
    got = gfe.echelon(A, 251)
    assert got["rank"] == 12000
    assert O.certify(A.cpu().numpy(), 251, host(got), nvec=4, seed=5) == 0
