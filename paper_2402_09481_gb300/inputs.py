"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no extractor arithmetic: it only draws bit strings and sizes.
It imports neither the CUDA binding nor the oracle, so both sides of every
parity test receive identical inputs from one place.

Generator: SplitMix64 in counter mode.  Word w of stream s is
``mix64(key_s + (w + 1) * 0x9E3779B97F4A7C15)`` with
``key_s = mix64(0x2402094810 ^ s)``, where ``mix64`` is the SplitMix64 output
function (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014).  With key 0 the counter stream is the classic
SplitMix64 sequence seeded with 0, which the tests check against its published
first outputs.

Bit strings are packed into uint64 words, bit i at word i >> 6, position i & 63
(least significant first); tail bits beyond the length are zero.
"""

from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
SEED_BASE = 0x2402094810

# P(bit = 1) = 0.8: bit = (u32 < ceil(0.8 * 2^32))
BIAS_08_THRESHOLD = 3435973837


def mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def stream_key(stream: int) -> np.uint64:
    return mix64(np.array([SEED_BASE ^ int(stream)], dtype=np.uint64))[0]


def counter_words(key, first: int, count: int) -> np.ndarray:
    """Words first .. first + count - 1 of the counter stream with this key."""
    w = np.arange(first + 1, first + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(np.uint64(key) + w * GAMMA)


def stream_words(stream: int, count: int, first: int = 0) -> np.ndarray:
    return counter_words(stream_key(stream), first, count)


def _mask_tail(words: np.ndarray, nbits: int) -> np.ndarray:
    tail = nbits & 63
    if tail and words.size:
        words[-1] &= np.uint64((1 << tail) - 1)
    return words


def bernoulli_half(stream: int, nbits: int) -> np.ndarray:
    """nbits i.i.d. Bernoulli(1/2) bits, packed (one generator word per 64 bits)."""
    nw = (nbits + 63) // 64
    out = np.empty(nw, dtype=np.uint64)
    step = 1 << 22
    for c in range(0, nw, step):
        out[c:c + step] = stream_words(stream, min(step, nw - c), first=c)
    return _mask_tail(out, nbits)


def bernoulli(stream: int, nbits: int, threshold_u32: int = BIAS_08_THRESHOLD) -> np.ndarray:
    """nbits i.i.d. bits with P(1) = threshold / 2^32, packed.

    Bit i uses the 32-bit half (i & 1) of generator word i >> 1 (low half
    first): bit = (u32 < threshold).
    """
    nw = (nbits + 63) // 64
    out = np.zeros(nw, dtype=np.uint64)
    step = 1 << 21  # words of output per chunk
    thr = np.uint64(threshold_u32)
    for c in range(0, nw, step):
        cw = min(step, nw - c)
        g = stream_words(stream, 32 * cw, first=32 * c).reshape(cw, 32)
        bits = np.empty((cw, 64), dtype=bool)
        bits[:, 0::2] = (g & np.uint64(0xFFFFFFFF)) < thr
        bits[:, 1::2] = (g >> np.uint64(32)) < thr
        # bit j of output word = bits[:, j] (little-endian bytes of the word)
        out[c:c + cw] = np.packbits(bits, axis=1, bitorder="little").view("<u8").reshape(cw)
    return _mask_tail(out, nbits)


def uniform01(stream: int, count: int, first: int = 0) -> np.ndarray:
    """count doubles in [0, 1) from the top 53 bits of each generator word."""
    w = stream_words(stream, count, first)
    return (w >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def loguniform_lengths(stream: int, count: int, lo_exp: float, hi_exp: float) -> np.ndarray:
    """n = floor(2^U), U ~ Uniform[lo_exp, hi_exp)."""
    u = uniform01(stream, count)
    return np.floor(np.exp2(lo_exp + (hi_exp - lo_exp) * u)).astype(np.int64)


def poisson_arrivals(stream: int, count: int, rate_per_s: float) -> np.ndarray:
    """Arrival times (s) of a Poisson process: cumulative exponential gaps."""
    u = uniform01(stream, count)
    gaps = -np.log1p(-u) / rate_per_s
    return np.cumsum(gaps)


def words_for(nbits: int) -> int:
    return (nbits + 63) // 64


def log2_ceil(v: int) -> int:
    return 0 if v <= 1 else int(math.ceil(math.log2(v)))
