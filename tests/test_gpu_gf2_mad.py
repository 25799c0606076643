"""The bit-packed GF(2) multiply-add (gfe_mad_gf2, Method of the Four
Russians tables) against the exact product mod 2 and against gfe_mad on
0/1 bytes (GPU)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1806_04211_gb300 import gfe, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def exact(W, A, B):
    """(W + A B) mod 2 on 0/1 byte matrices; float64 products are exact here."""
    P = (A.astype(np.float64) @ B.astype(np.float64)).astype(np.int64)
    if W is not None:
        P = P + W
    return (P % 2).astype(np.uint8)


@pytest.mark.parametrize("m,n,k,w", [(1, 1, 1, "none"), (3, 70, 65, "sep"), (1025, 1100, 200, "inplace"),
                                     (1500, 3000, 700, "sep"), (64, 64, 64, "none"), (2048, 1024, 4096, "inplace"),
                                     (300, 5000, 1, "sep"), (5000, 300, 129, "none"), (10, 20, 0, "sep")])
def test_mad_gf2_matches_exact_product(m, n, k, w):
    Aw = synth.bernoulli_gf2(m, max(k, 1), 31, 1)
    Bw = synth.bernoulli_gf2(max(k, 1), n, 31, 2)
    Ww = synth.bernoulli_gf2(m, n, 31, 3)
    A = O.unpack_bits(Aw.numpy(), k)
    B = O.unpack_bits(Bw.numpy(), n)[:k]
    W = O.unpack_bits(Ww.numpy(), n)
    Ad, Bd = Aw.to(DEV), Bw.to(DEV)
    if w == "none":
        C = gfe.mad_gf2(None, Ad, Bd, n, k)
        ref = exact(None, A, B)
    elif w == "sep":
        C = gfe.mad_gf2(Ww.to(DEV), Ad, Bd, n, k)
        ref = exact(W, A, B)
    else:
        C = Ww.to(DEV).clone()
        gfe.mad_gf2(C, Ad, Bd, n, k, out=C)
        ref = exact(W, A, B)
    got = C.cpu().numpy()
    assert np.array_equal(O.unpack_bits(got, n), ref)
    # pad bits beyond n in the last word are written 0
    nw = (n + 63) // 64
    assert np.array_equal(got.view(np.uint64)[:, :nw], O.pack_bits(ref, got.shape[1])[:, :nw])


def test_mad_gf2_equals_byte_mad():
    m, n, k = 3000, 2500, 1800
    Aw, Bw = synth.bernoulli_gf2(m, k, 5, 1), synth.bernoulli_gf2(k, n, 5, 2)
    A = torch.from_numpy(O.unpack_bits(Aw.numpy(), k)).to(DEV)
    B = torch.from_numpy(O.unpack_bits(Bw.numpy(), n)).to(DEV)
    C = gfe.mad_gf2(None, Aw.to(DEV), Bw.to(DEV), n, k)
    ref = gfe.mad(None, A, B, 2).cpu().numpy()
    assert np.array_equal(O.unpack_bits(C.cpu().numpy(), n), ref)


def test_gf2_peaks_are_plausible():
    pk = gfe.gf2_peaks()
    # LOP3: at most 152 SMs x 128 lanes x ~2.1 GHz; shared loads at most ~152 x 128 B x 2.1 GHz
    assert 1e13 < pk["lop3_per_s"] < 5e13
    assert 1e12 < pk["lds_bytes_per_s"] < 6e13
