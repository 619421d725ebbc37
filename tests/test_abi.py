"""CPU-side checks of the C ABI: the library loads, exports every declared
function, and its host logic (N_A primes, plans) agrees with the oracle and the
arithmetic of the middle-product form.  No GPU work is done here."""

import pytest

import oracle
from paper_2402_09481_gb300 import build, native


@pytest.fixture(scope="module")
def lib():
    build.build()
    return native.lib()


def test_exports_every_declared_function(lib):
    names = native.header_functions()
    assert len(names) >= 13
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding declares a prototype for each of them
    assert set(names) <= set(native.PROTOTYPES)


def test_status_strings(lib):
    for s in range(8):
        assert lib.cm_status_str(s).decode().startswith(native.STATUS[s])


def test_na_primes_match_oracle(lib):
    for P in range(0, 3000):
        assert native.is_na_prime(P) == oracle.has_primitive_root_2(P), P
    for n in (3, 100, 2 ** 20, 2 ** 24, 6500000001, 2 ** 32 + 5):
        assert native.next_na_prime(n) == oracle.next_na(n)
        assert native.prev_na_prime(n) == oracle.prev_na(n)
    assert native.next_na_prime(2 ** 24) == 16777259
    assert native.prev_na_prime(2 ** 30) == 1073741789


def test_plan_lengths(lib):
    T, C, D = native.TOEPLITZ, native.CIRCULANT, native.DODIS
    # smallest power of two >= K + m - 1
    assert native.ntt_length(T, 2 ** 16, 2 ** 15) == 2 ** 17
    assert native.ntt_length(C, 16777258, 8388629) == 2 ** 25
    assert native.ntt_length(D, 1073741789, 429496715) == 2 ** 31
    assert native.ntt_length(T, 1, 1) == 2
    assert native.ntt_length(T, 2 ** 31, 2 ** 31 + 1) == 2 ** 32
    # beyond one transform: blocked (here two output blocks of one transform each)
    assert native.ntt_length(T, 2 ** 31, 2 ** 31 + 2) == 2 ** 32
    # invalid: m = 0, n = 0, beyond 2^40, non-N_A lengths, m > n
    assert native.ntt_length(T, 2 ** 40 + 1, 5) == 0
    assert native.ntt_length(T, 5, 2 ** 40 + 1) == 0
    assert native.ntt_length(T, 5, 0) == 0
    assert native.ntt_length(T, 0, 5) == 0
    assert native.ntt_length(C, 6, 3) == 0      # 7 is prime but ord_7(2) = 3
    assert native.ntt_length(C, 10, 11) == 0    # m > n
    assert native.ntt_length(D, 9, 3) == 0      # 9 not prime
    assert native.ntt_length(D, 11, 12) == 0


def test_scratch_and_launches(lib):
    T, D = native.TOEPLITZ, native.DODIS
    assert native.scratch_bytes(T, 100, 50) == 0          # one CTA, no scratch
    assert native.launch_count(T, 100, 50) == 1
    L = 2 ** 17
    assert native.scratch_bytes(T, 2 ** 16, 2 ** 15) == 16 * L + 2 ** 15
    assert native.launch_count(T, 2 ** 16, 2 ** 15) == 5   # 2 fwd, middle, inv, pack
    assert native.launch_count(D, 1073741789, 429496715) == 9


def test_block_counts(lib):
    T, C, D = native.TOEPLITZ, native.CIRCULANT, native.DODIS
    assert native.block_count(T, 2 ** 16, 2 ** 15) == 1
    assert native.block_count(T, 2 ** 31, 2 ** 31 + 1) == 1
    # the QRNG example (n = 6.5e9, m = 581294933): K + m - 1 = 7.08e9 > 2^32,
    # input blocks of at most 2^32 - m + 1 = 3.71e9: two products
    assert native.block_count(T, 6_500_000_000, 581_294_933) == 2
    assert native.block_count(C, 6_500_000_068, 581_294_933) == 2
    # m above half the limit splits the output too: 2^12 limit, m = 3000 ->
    # output blocks of 2048, input blocks of at most 2049: 2 x 5
    assert native.block_count(T, 10_000, 3_000, 12) == 10
    assert native.block_count(T, 2000, 2000, 12) == 1
    assert native.block_count(T, 2000, 2098, 12) == 2
    assert native.block_count(T, 100, 50, 7) == 0
    assert native.block_count(T, 100, 50, 33) == 0
    assert native.block_count(T, 2 ** 40, 2 ** 40, 8) == 0     # over 65536 products
    assert native.block_count(C, 6, 3, 12) == 0                # 7 not in N_A
    # launches: both products plus one XOR pass
    one = native.launch_count(T, 2 ** 31, 2 ** 31 + 1)
    assert native.launch_count(T, 6_500_000_000, 581_294_933) == 2 * one + 1
