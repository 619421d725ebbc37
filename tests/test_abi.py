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
    # one transform: the smallest power of two >= K + m - 1
    assert native.ntt_length(T, 2 ** 16, 2 ** 15) == 2 ** 17
    assert native.plan_query(C, 16777258, 8388629, plan_mode=native.PLAN_SINGLE)["transform_length"] == 2 ** 25
    # the planner's form: two summed 2^24 products and an 83-term dense tail
    assert native.ntt_length(C, 16777258, 8388629) == 2 ** 24
    assert native.ntt_length(T, 1, 1) == 2
    assert native.ntt_length(T, 2 ** 31, 2 ** 31 + 1) == 2 ** 32
    # Dodis et al. at n = 2^30 runs as two 2^30 products over the 32-bit field
    # (estimated faster than one Goldilocks transform of 2^31, which single
    # mode keeps)
    assert native.ntt_length(D, 1073741789, 429496715) == 2 ** 30
    assert native.plan_query(D, 1073741789, 429496715, plan_mode=native.PLAN_SINGLE)["transform_length"] == 2 ** 31
    # one term beyond one transform: split into several products (here 2^30
    # products over the 32-bit field); single mode uses no dense tail
    q = native.plan_query(T, 2 ** 31, 2 ** 31 + 2)
    assert q["products"] > 1 and q["transform_length"] <= 2 ** 32
    s = native.plan_query(T, 2 ** 31, 2 ** 31 + 2, plan_mode=native.PLAN_SINGLE)
    assert s["products"] > 1 and s["tail_terms"] == 0
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
    # two operands of L 32-bit elements, then the parity bytes (held for the
    # column-pass form, which runs where the cluster kernel cannot)
    assert native.scratch_bytes(T, 2 ** 16, 2 ** 15) == 8 * L + 2 ** 15
    # one launch on a thread-block cluster of 16 CTAs
    assert native.launch_count(T, 2 ** 16, 2 ** 15) == 1
    # a longer transform: one forward pass (both operands), middle, inverse pass, pack
    assert native.launch_count(T, 2 ** 18, 2 ** 17) == 4
    # Dodis et al. at 2^30: precondition, then two summed products of two
    # column passes each: 2 x (2 fwd + middle) + 2 inv + pack
    assert native.launch_count(D, 1073741789, 429496715) == 1 + 2 * 3 + 3
    # Goldilocks, one transform of 2^31: precondition + 2 fwd + middle + 2 inv + pack
    single_gl = native.plan_query(D, 1073741789, 429496715, field=native.FIELD_GOLDILOCKS,
                                  plan_mode=native.PLAN_SINGLE)
    assert single_gl["launches"] == 7 and single_gl["scratch_bytes"] == 2 * 8 * 2 ** 31 + 429496832 + 256


def test_block_counts(lib):
    T, C, D = native.TOEPLITZ, native.CIRCULANT, native.DODIS
    assert native.block_count(T, 2 ** 16, 2 ** 15) == 1
    assert native.block_count(T, 2 ** 31, 2 ** 31 + 1) == 1
    # the QRNG example (n = 6.5e9, m = 581294933): K + m - 1 = 7.08e9 > 2^32;
    # 2^30 products over the 32-bit field, input blocks of at most
    # 2^30 - m + 1 = 492446892 terms: 14 products in one output window
    assert native.block_count(T, 6_500_000_000, 581_294_933) == 14
    assert native.block_count(C, 6_500_000_068, 581_294_933) == 14
    # 2^12 limit, m = 3000: two output windows of 1536 and 1464 rows and input
    # blocks of 2500 terms (2500 + 1536 - 1 <= 4096): 2 x 4, cheaper than one
    # window of 10 input blocks
    assert native.block_count(T, 10_000, 3_000, 12) == 8
    assert native.block_count(T, 2000, 2000, 12) == 1
    assert native.block_count(T, 2000, 2098, 12) == 2
    assert native.block_count(T, 100, 50, 7) == 0
    assert native.block_count(T, 100, 50, 33) == 0
    assert native.block_count(T, 2 ** 40, 2 ** 40, 8) == 0     # over 65536 products
    assert native.block_count(C, 6, 3, 12) == 0                # 7 not in N_A
    # launches: 14 forward halves (2 column passes + middle), three sum
    # groups (6, 6, 2) each with 2 inverse passes and a pack, two XOR passes
    assert native.launch_count(T, 6_500_000_000, 581_294_933) == 14 * 3 + 3 * 3 + 2
