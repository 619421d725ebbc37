"""Primes with 2 as a primitive root (the set N_A of the paper).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The Circulant construction (Def. ext-circ) needs its seed length, and the
Dodis et al. construction its input length, to be a prime P for which 2 is a
primitive root modulo P, i.e. the multiplicative order of 2 modulo P is P - 1.
This module decides that from the definition:

* ``is_prime``: Miller-Rabin with the first twelve prime bases, which is a
  proof of primality for every n < 3.3 * 10^24 (far above the 2^40 lengths
  the paper supports);
* ``has_primitive_root_2``: 2 generates (Z/PZ)^* iff 2^((P-1)/q) != 1 mod P
  for every prime q dividing P - 1 (q found by trial division);
* ``ord2_bruteforce``: the order of 2 by repeated doubling, for small P, used
  by the tests to pin ``has_primitive_root_2``;
* ``next_na`` / ``prev_na`` / ``closest_na``: the nearest members of N_A, in the
  spirit of the utility functions named in the footnote of Def. ext-circ.  On a
  tie ``closest_na`` takes the larger prime (the input is padded, not cut).
"""

from __future__ import annotations

_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(n: int) -> bool:
    if n < 2:
        return False
    for p in _MR_BASES:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def _prime_factors(n: int) -> list[int]:
    out = []
    q = 2
    while q * q <= n:
        if n % q == 0:
            out.append(q)
            while n % q == 0:
                n //= q
        q += 1 if q == 2 else 2
    if n > 1:
        out.append(n)
    return out


def has_primitive_root_2(P: int) -> bool:
    """True iff P is prime and 2 has multiplicative order P - 1 modulo P."""
    if P < 3 or not is_prime(P):
        return False
    return all(pow(2, (P - 1) // q, P) != 1 for q in _prime_factors(P - 1))


def ord2_bruteforce(P: int) -> int:
    """Multiplicative order of 2 modulo odd P > 1, by repeated doubling."""
    k, v = 1, 2 % P
    while v != 1:
        v = v * 2 % P
        k += 1
        if k > P:
            raise ValueError("2 is not invertible modulo P")
    return k


def next_na(n: int) -> int:
    """Smallest P >= n with P prime and 2 a primitive root modulo P."""
    P = max(n, 3)
    while not has_primitive_root_2(P):
        P += 1
    return P


def prev_na(n: int) -> int:
    """Largest P <= n with P prime and 2 a primitive root modulo P (n >= 3)."""
    if n < 3:
        raise ValueError("no member of N_A below 3")
    P = n
    while not has_primitive_root_2(P):
        P -= 1
    return P


def closest_na(n: int) -> int:
    """Member of N_A nearest to n; on a tie, the larger one."""
    up = next_na(n)
    if n < 3:
        return up
    down = prev_na(n)
    return up if up - n <= n - down else down
