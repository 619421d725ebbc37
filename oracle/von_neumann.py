"""Von Neumann deterministic extractor (Section "Von Neumann", Alg. vn).

TEST INFRASTRUCTURE ONLY (see the package docstring).

For j = 0 .. floor(n/2) - 1 the pair (x_{2j}, x_{2j+1}) yields the output bit
x_{2j} when the two bits differ and nothing when they are equal; the outputs
keep the order of j.  A trailing odd bit belongs to no pair and is ignored.

Alg. vn ends in an unconditional ``error`` step whose comment says the error is
for an input whose bits are all the same.  Reading: the extraction fails when it
produces no output bit at all (every pair equal, which includes the all-equal
input and inputs shorter than two bits); otherwise its output stands.

``von_neumann_loop`` is the definition as a plain loop (small inputs);
``von_neumann`` is the same selection written with array indexing, used at
larger sizes; ``tests/test_von_neumann_oracle.py`` pins one to the other and
both to hand-worked cases and to the unbiasedness property of the section.
"""

from __future__ import annotations

import numpy as np

from .extractors import pack_bits, unpack_bits


class VonNeumannNoOutput(ValueError):
    """Every pair of the input was equal: no output bit (the error of Alg. vn)."""


def von_neumann_loop(bits) -> list[int]:
    b = [int(v) & 1 for v in bits]
    out = []
    for j in range(len(b) // 2):
        if b[2 * j] != b[2 * j + 1]:
            out.append(b[2 * j])
    if not out:
        raise VonNeumannNoOutput("no pair of unequal bits")
    return out


def von_neumann(bits) -> np.ndarray:
    """uint8 0/1 input -> uint8 0/1 output, as ``von_neumann_loop``."""
    b = np.asarray(bits, dtype=np.uint8) & 1
    k = b.size // 2
    first, second = b[0:2 * k:2], b[1:2 * k:2]
    out = first[first != second]
    if out.size == 0:
        raise VonNeumannNoOutput("no pair of unequal bits")
    return out.copy()


def von_neumann_packed(words, n: int) -> tuple[np.ndarray, int]:
    """Packed input of n bits -> (packed output, output length m)."""
    out = von_neumann(unpack_bits(words, n))
    return pack_bits(out), int(out.size)


def pair_counts_per_word(words, n: int) -> np.ndarray:
    """Number of unequal pairs (x_{2j}, x_{2j+1}) that fall in each 64-bit word
    of the packed input (pairs never straddle a word; pairs past floor(n/2)
    do not count).  Written with word-wide bit operations so that inputs of
    billions of bits fit in memory: bit 2j of w ^ (w >> 1) is x_{2j} xor
    x_{2j+1}."""
    k = n // 2
    nw = (2 * k + 63) // 64
    w = np.asarray(words, dtype=np.uint64)[:nw].copy()
    if nw:
        vb = 2 * k - 64 * (nw - 1)
        if vb < 64:
            w[-1] &= np.uint64((1 << vb) - 1)
    d = (w ^ (w >> np.uint64(1))) & np.uint64(0x5555555555555555)
    if hasattr(np, "bitwise_count"):
        return np.bitwise_count(d).astype(np.int64)
    return np.array([bin(int(v)).count("1") for v in d], dtype=np.int64)


def output_bits_at(words, n: int, positions) -> tuple[np.ndarray, int]:
    """Output bits at the given output positions, and the output length m,
    without forming the whole output: the cumulative pair counts locate the
    word holding each position, and that word's pairs are filtered by the
    definition.  Positions must be < m."""
    cnt = pair_counts_per_word(words, n)
    cum = np.cumsum(cnt)
    m = int(cum[-1]) if cum.size else 0
    w = np.asarray(words, dtype=np.uint64)
    out = np.zeros(len(positions), dtype=np.uint8)
    for i, pos in enumerate(positions):
        pos = int(pos)
        if not 0 <= pos < m:
            raise IndexError(f"output position {pos} outside [0, {m})")
        wi = int(np.searchsorted(cum, pos, side="right"))
        before = int(cum[wi - 1]) if wi else 0
        npairs = min(32, n // 2 - 32 * wi)
        word = int(w[wi])
        local = []
        for j in range(npairs):
            a, b = (word >> (2 * j)) & 1, (word >> (2 * j + 1)) & 1
            if a != b:
                local.append(a)
        out[i] = local[pos - before]
    return out, m


def von_neumann_count(words, n: int) -> int:
    """Output length only (number of unequal pairs); 0 is allowed here."""
    b = unpack_bits(words, n)
    k = n // 2
    return int(np.count_nonzero(b[0:2 * k:2] != b[1:2 * k:2]))
