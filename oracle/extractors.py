"""Explicit-matrix GF(2) oracle for the three NTT-backed extractors.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product never imports
this module.

Bit strings: index 0 is the paper's x_0 (Section "Preliminaries").  Two encodings
are used here:

* unpacked: ``numpy.uint8`` arrays of 0/1, one bit per element;
* packed: ``numpy.uint64`` words, bit i at word ``i >> 6``, bit position
  ``i & 63`` (least significant first).  Tail bits past the length are zero on
  output and ignored on input.

Two tiers, both written from the definitions:

* ``*_matrix`` + ``gf2_matvec`` build the whole matrix entry by entry from the
  index formula and multiply modulo 2.  Used for small sizes.
* ``*_rows`` build only the requested rows, each as a packed bit vector (one
  row of the matrix, read off the same index formula, see ``_cyclic_rows``),
  and take the inner product with the other operand by AND + popcount.  Used at
  large sizes, where the full matrix does not fit in memory, to compute a
  sample of output bits.  Tests pin the second tier to the first.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "pack_bits", "unpack_bits", "toeplitz_matrix", "circulant_matrix",
    "dodis_matrix", "gf2_matvec", "toeplitz", "circulant", "dodis",
    "toeplitz_rows", "circulant_rows", "dodis_rows", "toeplitz_packed",
    "circulant_packed", "dodis_packed", "DodisPreconditionError",
]


class DodisPreconditionError(ValueError):
    """Dodis et al. needs x not all-zero and not all-one (Section "Dodis et al.")."""


# --------------------------------------------------------------------------- #
# bit packing
# --------------------------------------------------------------------------- #
def unpack_bits(words, nbits: int) -> np.ndarray:
    """Packed uint64 words (LSB first) -> uint8 0/1 array of length nbits."""
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint64))
    need = (nbits + 63) // 64
    if w.size < need:
        raise ValueError(f"need {need} words for {nbits} bits, got {w.size}")
    b = np.unpackbits(w[:need].astype("<u8").view(np.uint8), bitorder="little")
    return b[:nbits].copy()


def pack_bits(bits) -> np.ndarray:
    """uint8 0/1 array -> packed uint64 words (LSB first), tail bits zero."""
    b = np.asarray(bits, dtype=np.uint8)
    nbits = b.size
    nwords = (nbits + 63) // 64
    padded = np.zeros(nwords * 64, dtype=np.uint8)
    padded[:nbits] = b & 1
    return np.packbits(padded, bitorder="little").view("<u8").astype(np.uint64)


def _popcount_u64(a: np.ndarray) -> np.ndarray:
    if hasattr(np, "bitwise_count"):
        return np.bitwise_count(a)
    # Older numpy: count bits byte by byte.
    table = np.array([bin(i).count("1") for i in range(256)], dtype=np.uint8)
    return table[a.view(np.uint8)].reshape(a.shape + (8,)).sum(axis=-1)


# --------------------------------------------------------------------------- #
# tier 1: explicit matrices from the paper's index formulas
# --------------------------------------------------------------------------- #
def toeplitz_matrix(y, n: int, m: int) -> np.ndarray:
    """toep(y) of Eq. toep: an m x n matrix with T[i][j] = y[(i - j) mod (n+m-1)].

    The displayed matrix has first column y_0 .. y_{m-1} and first row
    y_0, y_{n+m-2}, ..., y_m; it has m rows and n columns (the text of
    Section "Toeplitz implementation" says so; the caption's "n x m" is read as
    rows x columns = m x n).
    """
    y = np.asarray(y, dtype=np.uint8)
    N = n + m - 1
    if y.size != N:
        raise ValueError("Toeplitz seed must have n + m - 1 bits")
    i = np.arange(m)[:, None]
    j = np.arange(n)[None, :]
    return y[(i - j) % N]


def circulant_matrix(c) -> np.ndarray:
    """circ(c) of Eq. circ-matrix: C[i][j] = c[(j - i) mod len(c)].

    Row 0 is c itself and row i is c right-shifted (cyclically) by i places.
    """
    c = np.asarray(c, dtype=np.uint8)
    P = c.size
    i = np.arange(P)[:, None]
    j = np.arange(P)[None, :]
    return c[(j - i) % P]


def dodis_matrix(x) -> np.ndarray:
    """The Dodis et al. matrix of Section "Dodis (and Circulant) implementation".

    Row 0 is x_0 .. x_{n-1}; row 1 is x_{n-1}, x_0, x_1, ...; in index form
    D[i][j] = x[(j - i) mod n].  Written out here from that display rather than
    by calling ``circulant_matrix``, so that a test can compare the two.
    """
    x = np.asarray(x, dtype=np.uint8)
    n = x.size
    D = np.empty((n, n), dtype=np.uint8)
    for i in range(n):
        for j in range(n):
            D[i, j] = x[(j - i) % n]
    return D


def gf2_matvec(M, v) -> np.ndarray:
    """(M v) mod 2 with exact integer accumulation."""
    M = np.asarray(M, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    return (M @ v & 1).astype(np.uint8)


def toeplitz(x, y, n: int, m: int) -> np.ndarray:
    """Toeplitz(x, y) = toep(y) x over GF(2) (Eq. toep-ext); unpacked bits."""
    x = np.asarray(x, dtype=np.uint8)
    if x.size != n:
        raise ValueError("Toeplitz input must have n bits")
    return gf2_matvec(toeplitz_matrix(y, n, m), x)


def circulant(x, y, n1: int, m: int) -> np.ndarray:
    """Circulant(x, y) of Def. ext-circ; unpacked bits.

    x has n1 = P - 1 bits and y has P bits, P prime with primitive root 2 (the
    caller's responsibility; the matrix product itself is defined for any P).
    x' = [x, 0] and the output is the first m entries of circ(x') y.
    """
    x = np.asarray(x, dtype=np.uint8)
    y = np.asarray(y, dtype=np.uint8)
    P = n1 + 1
    if x.size != n1 or y.size != P:
        raise ValueError("Circulant needs |x| = n1 and |y| = n1 + 1")
    if not 1 <= m <= n1:
        raise ValueError("Circulant needs 1 <= m <= n1")
    xp = np.concatenate([x, np.zeros(1, dtype=np.uint8)])
    return gf2_matvec(circulant_matrix(xp)[:m], y)


def dodis(x, y, n: int, m: int) -> np.ndarray:
    """Dodis(x, y): first m entries of D y (matrix form); unpacked bits."""
    x = np.asarray(x, dtype=np.uint8)
    y = np.asarray(y, dtype=np.uint8)
    if x.size != n or y.size != n:
        raise ValueError("Dodis needs |x| = |y| = n")
    if not 1 <= m <= n:
        raise ValueError("Dodis needs 1 <= m <= n")
    if x.min() == x.max():
        raise DodisPreconditionError("x is all-zero or all-one")
    return gf2_matvec(dodis_matrix(x)[:m], y)


# --------------------------------------------------------------------------- #
# tier 2: selected rows, each built as a packed bit vector
# --------------------------------------------------------------------------- #
def _doubled_packed(bits: np.ndarray) -> np.ndarray:
    """Packed words of the bit string bits || bits, plus one zero guard word."""
    w = pack_bits(np.concatenate([bits, bits]))
    return np.concatenate([w, np.zeros(2, dtype=np.uint64)])


def _cyclic_rows(gen_bits: np.ndarray, starts: np.ndarray, length: int,
                 other_words: np.ndarray, chunk_rows: int) -> np.ndarray:
    """Inner products <row_r, other> mod 2, row_r[j] = gen[(starts[r] + j) mod N].

    gen_bits has N bits; row r is the window of gen_bits read cyclically from
    position starts[r], ``length`` <= N bits long.  It is cut out of the packed
    doubled string with two shifts (the bits at positions s .. s + length - 1
    of gen || gen are exactly gen[(s + j) mod N] for s < N).
    """
    N = gen_bits.size
    W = _doubled_packed(gen_bits)
    nw = (length + 63) // 64
    other = np.asarray(other_words, dtype=np.uint64)[:nw].copy()
    tail = length - 64 * (nw - 1)
    if tail < 64:
        other[nw - 1] &= np.uint64((1 << tail) - 1)
    out = np.empty(starts.size, dtype=np.uint8)
    k = np.arange(nw + 1)
    for c0 in range(0, starts.size, chunk_rows):
        s = np.asarray(starts[c0:c0 + chunk_rows], dtype=np.int64) % N
        q = (s >> 6)[:, None]
        r = (s & 63).astype(np.uint64)[:, None]
        a = W[q + k[None, :]]
        lo = a[:, :-1] >> r
        hi = np.where(r == 0, np.uint64(0), a[:, 1:] << ((np.uint64(64) - r) & np.uint64(63)))
        win = lo | hi
        dots = _popcount_u64(win & other[None, :]).sum(axis=1)
        out[c0:c0 + chunk_rows] = (dots & 1).astype(np.uint8)
    return out


def _chunk_rows(length: int) -> int:
    # keep the gathered window block near 32 MiB
    return max(1, min(4096, (1 << 22) // ((length + 63) // 64 + 1)))


def toeplitz_rows(x_words, n: int, y_words, m: int, rows) -> np.ndarray:
    """Output bits z_i, i in rows, of Toeplitz(x, y) (Eq. toep-ext).

    z_i = sum_j y[(i - j) mod N] x_j.  Substituting j = n - 1 - t gives
    z_i = sum_t y[(i - n + 1 + t) mod N] * x_{n-1-t}, i.e. the cyclic window of
    y starting at (i - n + 1) mod N, of length n, against x reversed.
    """
    N = n + m - 1
    rows = np.asarray(rows, dtype=np.int64)
    if rows.size and (rows.min() < 0 or rows.max() >= m):
        raise ValueError("row index out of range")
    y = unpack_bits(y_words, N)
    xr = unpack_bits(x_words, n)[::-1]
    return _cyclic_rows(y, rows - (n - 1), n, pack_bits(xr), _chunk_rows(n))


def circulant_rows(x_words, n1: int, y_words, m: int, rows) -> np.ndarray:
    """Output bits z_i, i in rows, of Circulant(x, y) (Def. ext-circ).

    Row i of circ(x') is x'[(j - i) mod P] over j: the cyclic window of x'
    starting at (-i) mod P, of length P, against y.
    """
    P = n1 + 1
    rows = np.asarray(rows, dtype=np.int64)
    if not 1 <= m <= n1:
        raise ValueError("Circulant needs 1 <= m <= n1")
    if rows.size and (rows.min() < 0 or rows.max() >= m):
        raise ValueError("row index out of range")
    xp = np.concatenate([unpack_bits(x_words, n1), np.zeros(1, dtype=np.uint8)])
    return _cyclic_rows(xp, -rows, P, np.asarray(y_words, dtype=np.uint64), _chunk_rows(P))


def dodis_rows(x_words, y_words, n: int, m: int, rows) -> np.ndarray:
    """Output bits z_i, i in rows, of Dodis(x, y): row i is x[(j - i) mod n]."""
    rows = np.asarray(rows, dtype=np.int64)
    if not 1 <= m <= n:
        raise ValueError("Dodis needs 1 <= m <= n")
    if rows.size and (rows.min() < 0 or rows.max() >= m):
        raise ValueError("row index out of range")
    x = unpack_bits(x_words, n)
    if x.min() == x.max():
        raise DodisPreconditionError("x is all-zero or all-one")
    return _cyclic_rows(x, -rows, n, np.asarray(y_words, dtype=np.uint64), _chunk_rows(n))


def toeplitz_packed(x_words, n: int, y_words, m: int) -> np.ndarray:
    """All m output bits of Toeplitz(x, y), packed."""
    return pack_bits(toeplitz_rows(x_words, n, y_words, m, np.arange(m)))


def circulant_packed(x_words, n1: int, y_words, m: int) -> np.ndarray:
    """All m output bits of Circulant(x, y), packed."""
    return pack_bits(circulant_rows(x_words, n1, y_words, m, np.arange(m)))


def dodis_packed(x_words, y_words, n: int, m: int) -> np.ndarray:
    """All m output bits of Dodis(x, y), packed."""
    return pack_bits(dodis_rows(x_words, y_words, n, m, np.arange(m)))
