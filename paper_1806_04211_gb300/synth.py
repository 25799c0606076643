"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no echelonisation arithmetic.  It draws matrices over GF(p)
from a counter-based generator so that the same (seed, stream, index) gives the
same entry on the host and on the device:

  SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014): the output function
      z ^= z >> 30; z *= 0xBF58476D1CE4E5B9
      z ^= z >> 27; z *= 0x94D049BB133111EB
      z ^= z >> 31
  applied to  key(seed, stream) + (index + 1) * 0x9E3779B97F4A7C15  (mod 2^64),
  with key(seed, stream) = mix(seed * 0x9E3779B97F4A7C15 + stream * 0xD1B54A32D192ED03 + 1).

Entry (i, j) of an m x n matrix over GF(p) is  ((w & 0xFFFFFFFF) * p) >> 32  for
the word w at index i*n + j (uniform in [0, p) up to a bias below p / 2^32).
A GF(2) matrix is bit-packed: word c of row i is the word at index i*ldw + c,
with the bits at columns >= n cleared (ldw = words per row, rounded up to an
even count so that every row starts on a 16-byte boundary).

The paper's experiments use uniformly random matrices (Section 5); the
rank-deficient "twins" are products U*V mod p of uniform factors drawn on two
other streams.  The product is formed exactly with float32 matrix products
over chunks of the inner dimension short enough that no partial sum exceeds
2^24, reduced mod p after each chunk.

Everything is torch so the same code runs on the CPU (tests) and on the GPU
(large benchmark inputs).  torch int64 arithmetic wraps modulo 2^64; right
shifts are made logical with a mask.
"""
from __future__ import annotations

import torch

_MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
C1 = 0xBF58476D1CE4E5B9
C2 = 0x94D049BB133111EB
STREAM_MUL = 0xD1B54A32D192ED03


def _s64(x: int) -> int:
    """Python int -> the int64 with the same low 64 bits."""
    x &= _MASK64
    return x - (1 << 64) if x >> 63 else x


def mix64_int(z: int) -> int:
    """SplitMix64 output function on a Python int (reference, unsigned)."""
    z &= _MASK64
    z = ((z ^ (z >> 30)) * C1) & _MASK64
    z = ((z ^ (z >> 27)) * C2) & _MASK64
    return z ^ (z >> 31)


def stream_key(seed: int, stream: int) -> int:
    return mix64_int(seed * GAMMA + stream * STREAM_MUL + 1)


def word_int(seed: int, stream: int, index: int) -> int:
    """The generator's word at `index` as an unsigned Python int (reference)."""
    return mix64_int(stream_key(seed, stream) + (index + 1) * GAMMA)


def _lsr(z: torch.Tensor, s: int) -> torch.Tensor:
    return (z >> s) & ((1 << (64 - s)) - 1)


def words(seed: int, stream: int, start: int, count: int, device="cpu") -> torch.Tensor:
    """Words for indices start .. start+count-1 as int64 (two's complement)."""
    idx = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    z = idx * _s64(GAMMA) + _s64(stream_key(seed, stream))
    z = (z ^ _lsr(z, 30)) * _s64(C1)
    z = (z ^ _lsr(z, 27)) * _s64(C2)
    return z ^ _lsr(z, 31)


def _row_chunk(n: int) -> int:
    return max(1, (1 << 24) // max(n, 1))


def uniform_u8(m: int, n: int, p: int, seed: int, stream: int = 0, device="cpu") -> torch.Tensor:
    """m x n uint8 matrix, entries uniform in [0, p)."""
    out = torch.empty((m, n), dtype=torch.uint8, device=device)
    step = _row_chunk(n)
    for r0 in range(0, m, step):
        r1 = min(m, r0 + step)
        w = words(seed, stream, r0 * n, (r1 - r0) * n, device)
        out[r0:r1] = (((w & 0xFFFFFFFF) * p) >> 32).to(torch.uint8).view(r1 - r0, n)
    return out


def gf2_words_per_row(n: int) -> int:
    w = (n + 63) // 64
    return w + (w & 1)


def bernoulli_gf2(m: int, n: int, seed: int, stream: int = 0, device="cpu") -> torch.Tensor:
    """m x ldw int64 words: bit-packed uniform GF(2) matrix, pad bits zero."""
    ldw = gf2_words_per_row(n)
    out = words(seed, stream, 0, m * ldw, device).view(m, ldw)
    return mask_pad_gf2(out, n)


def mask_pad_gf2(wd: torch.Tensor, n: int) -> torch.Tensor:
    ldw = wd.shape[1]
    full, rem = divmod(n, 64)
    if full < ldw:
        if rem:
            wd[:, full] &= (1 << rem) - 1
            wd[:, full + 1:] = 0
        else:
            wd[:, full:] = 0
    return wd



def unpack_gf2(wd: torch.Tensor, n: int) -> torch.Tensor:
    """bit-packed words (m x ldw int64) -> m x n uint8 of 0/1 (rows in
    chunks, so the int64 temporaries stay near 1 GB)."""
    m, ldw = wd.shape
    out = torch.empty((m, n), dtype=torch.uint8, device=wd.device)
    sh = torch.arange(64, dtype=torch.int64, device=wd.device)
    step = max(1, (1 << 27) // (ldw * 64))
    for r0 in range(0, m, step):
        r1 = min(m, r0 + step)
        bits = ((wd[r0:r1].unsqueeze(-1) >> sh) & 1).to(torch.uint8).view(r1 - r0, ldw * 64)
        out[r0:r1] = bits[:, :n]
    return out


def pack_gf2(bits: torch.Tensor, ldw: int | None = None) -> torch.Tensor:
    """m x n uint8 of 0/1 -> m x ldw int64 words (bit c%64 of word c/64).
    Rows are packed in chunks so the int64 temporaries stay near 1 GB."""
    m, n = bits.shape
    if ldw is None:
        ldw = gf2_words_per_row(n)
    out = torch.empty((m, ldw), dtype=torch.int64, device=bits.device)
    sh = torch.arange(64, dtype=torch.int64, device=bits.device)
    step = max(1, (1 << 27) // (ldw * 64))
    for r0 in range(0, m, step):
        r1 = min(m, r0 + step)
        pad = torch.zeros((r1 - r0, ldw * 64), dtype=torch.int64, device=bits.device)
        pad[:, :n] = bits[r0:r1].to(torch.int64)
        out[r0:r1] = (pad.view(r1 - r0, ldw, 64) << sh).sum(-1)
    return out


def matmul_mod(U: torch.Tensor, V: torch.Tensor, p: int) -> torch.Tensor:
    """(U @ V) mod p for uint8 U, V with entries in [0, p), exactly.

    float32 products of chunks of the inner dimension short enough that every
    partial sum stays below 2^24 (so every float32 value is an exact integer),
    reduced mod p after each chunk.  Rows of U go in blocks, so the float32
    temporaries stay near 1 GB beside V's float32 copy."""
    m, k = U.shape
    n = V.shape[1]
    chunk = max(1, ((1 << 24) - 1) // max((p - 1) * (p - 1), 1))
    out = torch.empty((m, n), dtype=torch.uint8, device=U.device)
    rows = max(1, (1 << 28) // max(n, k, 1))
    old = None
    if U.is_cuda:
        old = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for k0 in range(0, max(k, 1), chunk):
            k1 = min(k, k0 + chunk)
            Vf = V[k0:k1].to(torch.float32)
            for r0 in range(0, m, rows):
                r1 = min(m, r0 + rows)
                prod = U[r0:r1, k0:k1].to(torch.float32) @ Vf
                acc = prod.to(torch.int32) if k0 == 0 else out[r0:r1].to(torch.int32) + prod.to(torch.int32)
                out[r0:r1] = (acc % p).to(torch.uint8)
            del Vf
    finally:
        if old is not None:
            torch.backends.cuda.matmul.allow_tf32 = old
    return out


def lowrank_u8(m: int, n: int, k: int, p: int, seed: int, device="cpu") -> torch.Tensor:
    """U(m x k) V(k x n) mod p with U, V uniform on streams 1 and 2 (rank <= k)."""
    U = uniform_u8(m, k, p, seed, 1, device)
    V = uniform_u8(k, n, p, seed, 2, device)
    return matmul_mod(U, V, p)


def lowrank_gf2(m: int, n: int, k: int, seed: int, device="cpu") -> torch.Tensor:
    """Bit-packed U V mod 2 with U, V uniform GF(2) on streams 1 and 2."""
    U = unpack_gf2(bernoulli_gf2(m, k, seed, 1, device), k)
    V = unpack_gf2(bernoulli_gf2(k, n, seed, 2, device), n)
    return pack_gf2(matmul_mod(U, V, 2))


def matrix(p: int, m: int, n: int, seed: int, rank: int | None = None, device="cpu") -> torch.Tensor:
    """The standard input: uniform (rank None) or a rank-deficient twin.

    GF(2) -> bit-packed int64 words (m x ldw); p > 2 -> uint8 (m x n)."""
    if p == 2:
        if rank is None:
            return bernoulli_gf2(m, n, seed, 0, device)
        return lowrank_gf2(m, n, rank, seed, device)
    if rank is None:
        return uniform_u8(m, n, p, seed, 0, device)
    return lowrank_u8(m, n, rank, p, seed, device)


PRIMES = [q for q in range(2, 252) if all(q % d for d in range(2, int(q ** 0.5) + 1))]


def c4_specs(count: int, seed: int = 1) -> list:
    """The batched workload's draw: (p, m, n, rank or None) per matrix, m and
    n log-uniform in [64, 2048] with aspect ratio <= 4 (resampled), p uniform
    in {2, 3, 5, 7}, every second matrix of rank 0.6 min(m, n).  Matrix i is
    drawn with matrix(p, m, n, seed=5000 + i, rank=rank)."""
    import numpy as np
    rng = np.random.RandomState(seed)
    out = []
    while len(out) < count:
        m, n = (int(round(64 * 32 ** rng.rand())) for _ in range(2))
        if max(m, n) > 4 * min(m, n):
            continue
        p = [2, 3, 5, 7][rng.randint(4)]
        rk = int(0.6 * min(m, n)) if len(out) % 2 else None
        out.append((p, m, n, rk))
    return out


def c5_specs(count: int, seed: int = 1) -> list:
    """The served workload's draw: (p, n, rank or None) per request, square n
    ~ Pareto(1.5) on [256, 16384] (rejection), p uniform over the primes
    <= 251, 30% of rank 0.6 n.  Request i is drawn with
    matrix(p, n, n, seed=7000 + i, rank=rank)."""
    import numpy as np
    rng = np.random.RandomState(seed)
    out = []
    while len(out) < count:
        n = 256 * (1 - rng.rand()) ** (-1 / 1.5)
        if n > 16384:
            continue
        n = int(n)
        p = PRIMES[rng.randint(len(PRIMES))]
        rk = int(0.6 * n) if rng.rand() < 0.3 else None
        out.append((p, n, rk))
    return out
