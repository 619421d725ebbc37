"""Pins of the RSH one-bit extractor oracle (oracle/trevisan.py).

Section "Trevisan implementation": l = ceil(log2 n + 2 log2(2/eps1)); chunks of
l bits as GF(2^l) elements, first bit most significant; p(x) = sum_i x_i
alpha1^(s-i) (Eq. poly); output = GF(2) inner product of alpha2 and p(x).
Every check below is fixed by mathematics or by the paper's text, not by the
oracle itself: the number of irreducible polynomials of each degree (Gauss's
formula) and brute-force factoring, the field laws and Fermat's little theorem
in GF(2^l), the paper's chunk example, a hand-worked extraction, and the exact
collision count of a polynomial hash followed by a Hadamard code.
"""

import itertools
import math

import numpy as np
import pytest

from oracle import trevisan as tv


def mobius(n):
    res, p, m = 1, 2, n
    while p * p <= m:
        if m % p == 0:
            m //= p
            if m % p == 0:
                return 0
            res = -res
        p += 1
    return -res if m > 1 else res


def n_irreducible(l):
    """Gauss: (1/l) sum_{d | l} mu(d) 2^(l/d)."""
    return sum(mobius(d) * 2 ** (l // d) for d in range(1, l + 1) if l % d == 0) // l


def irreducible_brute(f):
    """No factor of degree 1 .. deg/2 (trial division over every polynomial)."""
    l = f.bit_length() - 1
    for g in range(2, 1 << (l // 2 + 1)):
        if g.bit_length() - 1 >= 1 and tv.poly_mod(f, g) == 0 and g != f:
            return False
    return l >= 1


@pytest.mark.parametrize("l", range(1, 11))
def test_irreducible_count_gauss(l):
    got = sum(1 for f in range(1 << l, 1 << (l + 1)) if tv.is_irreducible(f))
    assert got == n_irreducible(l)


def test_rabin_matches_trial_division():
    for f in range(2, 1 << 10):
        assert tv.is_irreducible(f) == irreducible_brute(f), bin(f)


@pytest.mark.parametrize("l", range(2, 13))
def test_modulus_is_first_in_documented_order(l):
    top = 1 << l
    cands = [top | (1 << k) | 1 for k in range(1, l)]
    cands += [top | (1 << a) | (1 << b) | (1 << c) | 1
              for a in range(3, l) for b in range(2, a) for c in range(1, b)]
    first = next(f for f in cands if irreducible_brute(f))
    assert tv.rsh_modulus(l) == first


def test_modulus_known_values():
    assert tv.rsh_modulus(3) == 0b1011            # x^3 + x + 1
    assert tv.rsh_modulus(4) == 0b10011           # x^4 + x + 1
    # no irreducible trinomial has degree 8 (all are reducible): a pentanomial
    f8 = tv.rsh_modulus(8)
    assert bin(f8).count("1") == 5 and irreducible_brute(f8)
    assert not any(irreducible_brute((1 << 8) | (1 << k) | 1) for k in range(1, 8))


@pytest.mark.parametrize("l", [8, 13, 64, 102, 127])
def test_field_laws_and_fermat(l):
    f = tv.rsh_modulus(l)
    rng = np.random.default_rng(l)
    for _ in range(5):
        a, b, c = (int.from_bytes(rng.bytes(32), "little") & ((1 << l) - 1) for _ in range(3))
        assert tv.gf_mul(a, tv.gf_mul(b, c, f), f) == tv.gf_mul(tv.gf_mul(a, b, f), c, f)
        assert tv.gf_mul(a, b ^ c, f) == tv.gf_mul(a, b, f) ^ tv.gf_mul(a, c, f)
        assert tv.gf_mul(a, b, f) == tv.gf_mul(b, a, f)
        if a:
            assert tv.gf_pow(a, (1 << l) - 1, f) == 1   # the multiplicative group has order 2^l - 1
    assert tv.gf_mul(1, 0b1011, f) == 0b1011


def test_field_bits_formula():
    # l = ceil(log2 n + 2 log2(2 / eps1))
    assert tv.rsh_field_bits(2 ** 20, 2.0 ** -40) == 20 + 2 * 41
    assert tv.rsh_field_bits(1000, 1e-10) == math.ceil(math.log2(1000) + 2 * math.log2(2e10))


def test_paper_chunk_example():
    # "if l = 3 and x0 = {0, 0, 1} then x0 = 1 in GF(2^3)"
    assert tv.element([0, 0, 1], 0, 3) == 1
    assert tv.element([1, 0, 0], 0, 3) == 4
    # chunks are cut in order and the last one is padded with 0s
    assert tv.chunks([1, 1, 0, 1, 0], 5, 3) == [0b110, 0b100]


def test_hand_worked_extraction():
    # l = 3, f = x^3 + x + 1; x = 101 011: x1 = x^2 + 1, x2 = x + 1;
    # alpha1 = 010 = x, alpha2 = 110 = x^2 + x.
    # p = x1 alpha1 + x2 = (x^3 + x) + (x + 1) = x^3 + 1 = (x + 1) + 1 = x,
    # and alpha2 . p = (0,1,1) . (0,1,0) over the coefficients of x^0, x^1, x^2 = 1.
    x = [1, 0, 1, 0, 1, 1]
    seed = [0, 1, 0, 1, 1, 0]
    assert tv.rsh_poly([0b101, 0b011], 0b010, 0b1011) == 0b010
    assert tv.rsh_onebit(x, 6, seed, 3) == 1
    assert tv.rsh_onebit(x, 6, [0, 1, 0, 1, 0, 1], 3) == 0   # alpha2 = 101 misses p = 010


@pytest.mark.parametrize("l,s", [(5, 4), (16, 9), (61, 30)])
def test_horner_equals_sum_of_powers(l, s):
    f = tv.rsh_modulus(l)
    rng = np.random.default_rng(100 + l)
    xs = [int(v) for v in rng.integers(0, 1 << min(l, 62), size=s)]
    a = int(rng.integers(1, 1 << min(l, 62)))
    assert tv.rsh_poly(xs, a, f) == tv.rsh_poly_powers(xs, a, f)


def test_linearity_in_x():
    rng = np.random.default_rng(7)
    n, l = 300, 23
    for _ in range(10):
        x1 = rng.integers(0, 2, n)
        x2 = rng.integers(0, 2, n)
        seed = rng.integers(0, 2, 2 * l)
        z = tv.rsh_onebit(x1 ^ x2, n, seed, l)
        assert z == tv.rsh_onebit(x1, n, seed, l) ^ tv.rsh_onebit(x2, n, seed, l)
    assert tv.rsh_onebit(np.zeros(n, dtype=np.uint8), n, rng.integers(0, 2, 2 * l), l) == 0


def test_collision_count_exact():
    # x != x': over all (alpha1, alpha2), z(x) = z(x') exactly when alpha1 is
    # a root of the difference polynomial D (then every alpha2 collides), or
    # for half of the alpha2 otherwise (a nonzero vector's inner products are
    # balanced): count = R 2^l + (2^l - R) 2^(l-1), R = #roots <= s - 1.
    l, s = 4, 3
    n = l * s
    f = tv.rsh_modulus(l)
    rng = np.random.default_rng(11)
    for _ in range(4):
        x = rng.integers(0, 2, n)
        xp = x.copy()
        xp[rng.integers(0, n)] ^= 1
        d = [a ^ b for a, b in zip(tv.chunks(x, n, l), tv.chunks(xp, n, l))]
        R = sum(1 for a in range(1 << l) if tv.rsh_poly_powers(d, a, f) == 0)
        assert R <= s - 1
        count = 0
        for a1, a2 in itertools.product(range(1 << l), repeat=2):
            seed = [(a1 >> (l - 1 - j)) & 1 for j in range(l)] + [(a2 >> (l - 1 - j)) & 1 for j in range(l)]
            count += tv.rsh_onebit(x, n, seed, l) == tv.rsh_onebit(xp, n, seed, l)
        assert count == R * 2 ** l + (2 ** l - R) * 2 ** (l - 1)


def test_trevisan_gathers_sets_in_increasing_order():
    rng = np.random.default_rng(5)
    n, l, d, m = 200, 9, 120, 7
    x = rng.integers(0, 2, n)
    y = rng.integers(0, 2, d)
    sets = [rng.choice(d, 2 * l + 3, replace=False) for _ in range(m)]
    out = tv.trevisan(x, n, y, sets, l)
    for i, S in enumerate(sets):
        assert out[i] == tv.rsh_onebit(x, n, y[np.sort(S)], l)
    with pytest.raises(ValueError):
        tv.trevisan(x, n, y, [np.arange(2 * l - 1)], l)
