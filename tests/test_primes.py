"""Pins for the oracle's N_A prime generator (primes with primitive root 2)."""

import os

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_pins():
    out = {}
    with open(os.path.join(GOLDEN, "paper_pins.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                out[k] = int(v)
    return out


def test_has_primitive_root_2_vs_bruteforce_order():
    for P in range(3, 2000):
        expect = oracle.is_prime(P) and oracle.ord2_bruteforce(P) == P - 1
        assert oracle.has_primitive_root_2(P) == expect, P


def test_is_prime_vs_sieve():
    N = 20000
    sieve = [True] * N
    sieve[0] = sieve[1] = False
    for i in range(2, int(N ** 0.5) + 1):
        if sieve[i]:
            for j in range(i * i, N, i):
                sieve[j] = False
    assert all(oracle.is_prime(i) == sieve[i] for i in range(N))
    # strong pseudoprimes to several small bases are rejected
    for c in (3215031751, 2152302898747, 3474749660383, 341550071728321):
        assert not oracle.is_prime(c)


def test_na_set_head():
    with open(os.path.join(GOLDEN, "na_set_head.txt")) as f:
        head = [int(t) for line in f if not line.startswith("#") for t in line.split()]
    got = [p for p in range(3, head[-1] + 1) if oracle.has_primitive_root_2(p)]
    assert got == head


def test_paper_qrng_pins():
    pins = read_pins()
    # Toeplitz seed length n_2 = n_1 + m - 1 (Section "Toeplitz")
    assert pins["toeplitz_n1"] + pins["toeplitz_m"] - 1 == pins["toeplitz_n2"]
    P = oracle.closest_na(pins["circulant_target"])
    assert P == pins["circulant_prime"]
    assert pins["toeplitz_n2"] - P == pins["circulant_seed_saving"]
    assert oracle.prev_na(pins["circulant_target"]) == 6499999931
    assert oracle.next_na(pins["circulant_target"]) == P


def test_next_prev_at_workload_sizes():
    # the sizes the benchmark uses: smallest member >= 2^24 (Circulant seed
    # length) and largest member <= 2^30 (Dodis length)
    P = oracle.next_na(2 ** 24)
    assert P == 16777259 and oracle.has_primitive_root_2(P)
    assert all(not oracle.has_primitive_root_2(q) for q in range(2 ** 24, P))
    Q = oracle.prev_na(2 ** 30)
    assert Q == 1073741789
    assert all(not oracle.has_primitive_root_2(q) for q in range(Q + 1, 2 ** 30 + 1))
