"""The bit-packed CPU NTT baseline (cpu_ntt/) against the oracle, CPU only.

The baseline computes the same extractions by its own code (the paper's field
of 3 * 2^30 + 1, radix-2 transforms with Shoup products, threads); its output
must equal the oracle's bit for bit: full outputs at small and medium sizes,
ragged lengths, m = 1 and maximal m, sampled rows at a transform of 2^22, and
the same bits for 1 and several threads.
"""

import numpy as np
import pytest

import cpu_ntt
import oracle
from paper_2402_09481_gb300 import inputs

T, C, D = cpu_ntt.TOEPLITZ, cpu_ntt.CIRCULANT, cpu_ntt.DODIS


def resolve(kind, n, m):
    if isinstance(n, str):
        P = oracle.next_na(int(n[1:]))
        n = P - 1 if kind == C else P
        m = max(1, int(m * n))
    return n, m


def ybits(kind, n, m):
    return n + m - 1 if kind == T else (n + 1 if kind == C else n)


def want(kind, xw, n, yw, m):
    if kind == T:
        return oracle.toeplitz_packed(xw, n, yw, m)
    if kind == C:
        return oracle.circulant_packed(xw, n, yw, m)
    return oracle.dodis_packed(xw, yw, n, m)


CASES = [(T, 1, 1), (T, 5, 3), (T, 64, 64), (T, 1000, 1000), (T, 8191, 8194), (T, 20000, 12001),
         (T, 100000, 31073), (C, "P3", 1.0), (C, "P5000", 0.5), (C, "P40000", 0.9), (C, "P131101", 0.5),
         (D, "P11", 0.5), (D, "P3000", 0.9), (D, "P40000", 0.4), (D, "P9000", 1.0)]


@pytest.mark.parametrize("kind,n,m", CASES)
def test_cpu_ntt_matches_oracle(kind, n, m):
    n, m = resolve(kind, n, m)
    xw = inputs.bernoulli_half(40 + n % 37, n)
    if kind == D:
        xw[0] = (xw[0] | np.uint64(1)) & ~np.uint64(2)
    yw = inputs.bernoulli_half(41 + m % 31, ybits(kind, n, m))
    w = want(kind, xw, n, yw, m)
    for threads in (1, 3):
        assert (cpu_ntt.extract(kind, xw, n, yw, m, threads) == w).all(), (kind, n, m, threads)


def test_cpu_ntt_sampled_rows_at_2_22():
    # Circulant, P = next N_A prime above 2^21, m = P - 1 (K + m - 1 near 2^22)
    P = oracle.next_na(2 ** 21)
    n, m = P - 1, P - 1
    xw, yw = inputs.bernoulli_half(50, n), inputs.bernoulli_half(51, n + 1)
    z = cpu_ntt.extract(C, xw, n, yw, m, 4)
    rows = np.unique(np.concatenate([np.arange(16), np.arange(m - 16, m),
                                     np.random.default_rng(9).integers(0, m, 48)]))
    got = ((z[rows >> 6] >> (rows & 63).astype(np.uint64)) & np.uint64(1)).astype(np.uint8)
    assert (got == oracle.circulant_rows(xw, n, yw, m, rows)).all()
    if m & 63:
        assert int(z[-1]) >> (m & 63) == 0


def test_cpu_ntt_rejects():
    z = np.zeros(4, dtype=np.uint64)
    for kind, n, m in [(C, 8, 3), (D, 9, 3), (C, 10, 11), (T, 5, 0), (T, 0, 5), (T, 2 ** 29 + 1, 2 ** 29 + 1)]:
        with pytest.raises(ValueError):
            cpu_ntt.extract(kind, z, n, z, m)  # 9 not prime; m > n; empty; beyond 2^30
