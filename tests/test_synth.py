"""The seeded input generator (CPU)."""
import numpy as np
import torch

from paper_1806_04211_gb300 import synth
from oracle import oracle as O


def test_splitmix64_published_vector():
    # SplitMix64 with state 0: first outputs (Steele, Lea, Flood 2014 reference code)
    g = synth.GAMMA
    assert synth.mix64_int(g) == 0xE220A8397B1DCDAF
    assert synth.mix64_int(2 * g) == 0x6E789E6AA1B965F4
    assert synth.mix64_int(3 * g) == 0x06C45D188009454F


def test_torch_words_match_reference():
    w = synth.words(7, 3, 100, 50)
    for k in range(50):
        assert (int(w[k]) & ((1 << 64) - 1)) == synth.word_int(7, 3, 100 + k)


def test_uniform_u8_range_and_determinism():
    a = synth.uniform_u8(37, 41, 7, seed=5)
    b = synth.uniform_u8(37, 41, 7, seed=5)
    assert a.dtype == torch.uint8 and torch.equal(a, b)
    assert int(a.max()) < 7
    w = synth.word_int(5, 0, 3 * 41 + 4)
    assert int(a[3, 4]) == ((w & 0xFFFFFFFF) * 7) >> 32
    counts = np.bincount(a.numpy().ravel(), minlength=7)
    assert counts.min() > 0


def test_gf2_pad_bits_zero_and_pack_roundtrip():
    W = synth.bernoulli_gf2(9, 70, seed=2)
    assert W.shape == (9, 2)
    assert int((W[:, 1] >> 6).abs().sum()) == 0
    bits = synth.unpack_gf2(W, 70)
    assert torch.equal(synth.pack_gf2(bits), W)
    assert np.array_equal(O.unpack_bits(W.numpy(), 70), bits.numpy())


def test_matmul_mod_exact():
    for p in (2, 3, 251):
        U = synth.uniform_u8(20, 700, p, 1, 1)
        V = synth.uniform_u8(700, 30, p, 1, 2)
        ref = (U.numpy().astype(np.int64) @ V.numpy().astype(np.int64)) % p
        assert np.array_equal(synth.matmul_mod(U, V, p).numpy(), ref)


def test_lowrank_twin_rank():
    A = synth.lowrank_u8(60, 50, 30, 251, seed=1)
    assert O.echelon(A.numpy(), 251)["rank"] == 30
    W = synth.lowrank_gf2(60, 70, 20, seed=1)
    assert O.echelon_gf2(W.numpy(), 60, 70)["rank"] <= 20
