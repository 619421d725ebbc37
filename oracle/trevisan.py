"""Trevisan's extractor, one-bit step: the Reed-Solomon-Hadamard (RSH) one-bit
extractor of Section "Trevisan implementation" (subsection of the appendix).

TEST INFRASTRUCTURE ONLY (see the package docstring): plain Python integers,
one bit at a time where that is clearest.

What the paper fixes:
- l = ceil(log2(n) + 2 log2(2 / eps1)) (rsh_field_bits);
- the input x is cut into s = ceil(n / l) chunks of l bits, the last padded
  with 0s; each chunk is an element of GF(2^l) by its binary representation,
  the first listed bit the most significant (the paper's example: l = 3,
  x0 = {0, 0, 1} is the element 1);
- alpha1 is the element given by the first l bits of the one-bit extractor's
  seed, alpha2 by the next l bits (same representation);
- p(x) = sum_{i=1..s} x_i alpha1^(s - i) over GF(2^l) (Eq. poly), and the
  output bit is the GF(2) inner product of the coefficient vectors of alpha2
  and p(x);
- Trevisan(x, y)_i = Ext1(x, y_{S_i}) for the weak design's sets S_i
  (y_{S_i}: the bits of y at the indices of S_i).

Readings (the paper is silent):
- the GF(2^l) modulus: the irreducible trinomial x^l + x^k + 1 with the
  smallest k, else the irreducible pentanomial x^l + x^a + x^b + x^c + 1
  (l > a > b > c > 0) with the smallest (a, b, c) in lexicographic order
  (rsh_modulus);
- y_{S_i} lists the bits of y at the indices of S_i in increasing order;
- the weak design itself (the block weak design of Mauerer et al., which the
  paper cites but does not state) is an input: the sets S_i are given.

Pinned by tests/test_trevisan_oracle.py: the modulus against brute-force
factoring for small l, the field laws, Horner against the explicit sum of
powers, GF(2)-linearity, the paper's chunk example, a hand-worked extraction,
and the exact collision counts of the polynomial-hash + Hadamard construction
against brute force.
"""

from __future__ import annotations

import math

import numpy as np

# --------------------------------------------------------------------------- #
# GF(2)[x] with Python integers (bit k = coefficient of x^k)
# --------------------------------------------------------------------------- #


def clmul(a: int, b: int) -> int:
    """Carry-less product of two GF(2)[x] polynomials."""
    r = 0
    while b:
        if b & 1:
            r ^= a
        a <<= 1
        b >>= 1
    return r


def poly_mod(a: int, f: int) -> int:
    """a mod f in GF(2)[x]."""
    df = f.bit_length() - 1
    while a and a.bit_length() - 1 >= df:
        a ^= f << (a.bit_length() - 1 - df)
    return a


def poly_gcd(a: int, b: int) -> int:
    while b:
        a, b = b, poly_mod(a, b)
    return a


def _x_pow_2k_mod(k: int, f: int) -> int:
    """x^(2^k) mod f by k squarings."""
    r = 0b10
    for _ in range(k):
        r = poly_mod(clmul(r, r), f)
    return r


def _prime_factors(n: int) -> list[int]:
    out, p = [], 2
    while p * p <= n:
        if n % p == 0:
            out.append(p)
            while n % p == 0:
                n //= p
        p += 1
    if n > 1:
        out.append(n)
    return out


def is_irreducible(f: int) -> bool:
    """Rabin's test for f of degree l >= 1: x^(2^l) = x mod f, and
    gcd(x^(2^(l/r)) - x, f) = 1 for every prime r dividing l."""
    l = f.bit_length() - 1
    if l < 1:
        return False
    if _x_pow_2k_mod(l, f) != poly_mod(0b10, f):
        return False
    for r in _prime_factors(l):
        if poly_gcd(_x_pow_2k_mod(l // r, f) ^ 0b10, f) != 1:
            return False
    return True


def rsh_modulus(l: int) -> int:
    """The GF(2^l) modulus (the reading above), as an integer with bit l set."""
    if l < 2:
        raise ValueError("l >= 2")
    top = 1 << l
    for k in range(1, l):
        f = top | (1 << k) | 1
        if is_irreducible(f):
            return f
    for a in range(3, l):
        for b in range(2, a):
            for c in range(1, b):
                f = top | (1 << a) | (1 << b) | (1 << c) | 1
                if is_irreducible(f):
                    return f
    raise ValueError(f"no irreducible trinomial or pentanomial of degree {l}")


def gf_mul(a: int, b: int, f: int) -> int:
    """Product in GF(2)[x] / f."""
    return poly_mod(clmul(a, b), f)


def gf_pow(a: int, e: int, f: int) -> int:
    r = 1
    while e:
        if e & 1:
            r = gf_mul(r, a, f)
        a = gf_mul(a, a, f)
        e >>= 1
    return r


# --------------------------------------------------------------------------- #
# RSH one-bit extractor
# --------------------------------------------------------------------------- #


def rsh_field_bits(n: int, eps1: float) -> int:
    """l = ceil(log2(n) + 2 log2(2 / eps1))."""
    return math.ceil(math.log2(n) + 2 * math.log2(2.0 / eps1))


def element(bits, start: int, l: int) -> int:
    """GF(2^l) element from l bits starting at `start` (0 past the end), the
    first bit the most significant coefficient."""
    v = 0
    for j in range(l):
        b = int(bits[start + j]) if start + j < len(bits) else 0
        v = (v << 1) | b
    return v


def chunks(x_bits, n: int, l: int) -> list[int]:
    """x_1 .. x_s: the input cut into s = ceil(n / l) chunks of l bits."""
    s = -(-n // l)
    xb = np.asarray(x_bits[:n], dtype=np.uint8)
    return [element(xb, i * l, l) for i in range(s)]


def rsh_poly(xs: list[int], alpha1: int, f: int) -> int:
    """p(x) = sum_i x_i alpha1^(s - i), by Horner's rule."""
    p = 0
    for c in xs:
        p = gf_mul(p, alpha1, f) ^ c
    return p


def rsh_poly_powers(xs: list[int], alpha1: int, f: int) -> int:
    """The same sum with every power computed on its own (a check of Horner)."""
    s = len(xs)
    acc = 0
    for i, c in enumerate(xs, start=1):
        acc ^= gf_mul(c, gf_pow(alpha1, s - i, f), f)
    return acc


def rsh_onebit(x_bits, n: int, seed_bits, l: int, f: int | None = None) -> int:
    """Ext1(x, seed): alpha1 = seed[0:l], alpha2 = seed[l:2l]; the parity of the
    coefficient-wise AND of alpha2 and p(x)."""
    f = rsh_modulus(l) if f is None else f
    a1 = element(seed_bits, 0, l)
    a2 = element(seed_bits, l, l)
    p = rsh_poly(chunks(x_bits, n, l), a1, f)
    return bin(a2 & p).count("1") & 1


def trevisan(x_bits, n: int, y_bits, sets, l: int) -> np.ndarray:
    """Trevisan(x, y)_i = Ext1(x, y_{S_i}), i < m = len(sets); each S_i a set of
    at least 2l indices into y (read in increasing order)."""
    f = rsh_modulus(l)
    xs = chunks(x_bits, n, l)
    y = np.asarray(y_bits, dtype=np.uint8)
    out = np.zeros(len(sets), dtype=np.uint8)
    for i, S in enumerate(sets):
        sub = y[np.sort(np.asarray(S, dtype=np.int64))]
        if sub.size < 2 * l:
            raise ValueError("every set needs at least 2l indices")
        a1, a2 = element(sub, 0, l), element(sub, l, l)
        out[i] = bin(a2 & rsh_poly(xs, a1, f)).count("1") & 1
    return out
