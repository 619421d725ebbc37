"""Host side of the Trevisan one-bit step: the library's GF(2^l) modulus
search and field-size formula against the oracle (CPU only)."""

import math

import pytest

from oracle import trevisan as tv
from paper_2402_09481_gb300 import native


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2402_09481_gb300 import build
    build.build()


def taps_of(f, l):
    return sorted((k for k in range(1, l) if (f >> k) & 1), reverse=True)


@pytest.mark.parametrize("l", list(range(2, 70)) + [100, 102, 121, 127, 128])
def test_modulus_matches_oracle(l):
    assert native.rsh_modulus(l) == taps_of(tv.rsh_modulus(l), l)


def test_modulus_limits():
    for l in (0, 1, 257):
        with pytest.raises(native.CMError):
            native.rsh_modulus(l)
    assert native.rsh_modulus(256) == [10, 5, 2]    # x^256 + x^10 + x^5 + x^2 + 1


def test_field_bits():
    for n, e in ((2 ** 20, 2.0 ** -40), (1000, 1e-10), (6_500_000_000, 1e-12), (2, 0.5)):
        assert native.rsh_field_bits(n, e) == tv.rsh_field_bits(n, e) == math.ceil(math.log2(n) + 2 * math.log2(2 / e))
    assert native.rsh_field_bits(0, 0.1) == 0 and native.rsh_field_bits(10, 0.0) == 0
    assert native.rsh_field_bits(10, 1.0) == 0


def test_every_modulus_has_small_taps():
    # the GPU reduction multiplies by x^l mod f with shifts in two rounds,
    # which needs 2 t_max - 2 < l for the largest middle exponent t_max
    for l in range(2, 257):
        assert 2 * max(native.rsh_modulus(l)) < l + 2, l
