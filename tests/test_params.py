"""The parameter layer: output lengths, Trevisan seed lengths, N_A planning.

Part 1 pins the oracle (oracle/params.py) to things other than itself:
the arithmetic the paper prints for its QKD and QRNG examples; each closed-form
two-source and Markov-model bound re-derived here from the base theorem it
comes from (the seeded bound of Thm. circSEED / the Toeplitz theorem, the
classical Dodis et al. two-source bound, the seeded Trevisan bound) and the
error transformations of Thm. 2-weak-source, Thm. Markov1 and Thm. Markov2;
special cases where a two-source bound must fall back to the seeded one; a
hand-worked Trevisan seed length; monotonicity.

Part 2 checks the C ABI (cm_output_length, cm_trevisan_seed_length,
cm_plan_params, cm_closest_na_prime) against the oracle on seeded random
parameters, and its argument checks.  All of it is host arithmetic: no GPU.
"""

import math

import numpy as np
import pytest

import oracle
from oracle import params as P

LE10 = math.log2(1e-10)     # the examples' epsilon = 10^-10
LOG3 = math.log2(3.0)


# ----- Part 1: pins of the oracle ------------------------------------------

def test_qrng_example_printed_numbers():
    # Section "Cryptomite for randomness extraction in (Q)RNG": min-entropy
    # rate 0.08943 of n1 = 6.5e9 bits, eps = 1e-10, Toeplitz:
    k1 = math.floor(0.08943 * 6.5e9)
    assert k1 == 581295000
    p = P.plan("toeplitz", "seeded", "quantum", 6500000000, k1, LE10)
    assert p["m"] == 581294933
    assert p["n2"] == 7081294932 == 6500000000 + 581294933 - 1
    # the Circulant extension: closest N_A member to n1 + 1 is 6.5e9 + 69, the
    # input padded by 68 fixed bits, the same m, 581294863 seed bits saved
    c = P.plan("circulant", "seeded", "quantum", 6500000000, k1, LE10, adjust="closest")
    assert c["n2"] == 6500000069 and c["n1"] == 6500000068 and c["pad_input"] == 68
    assert c["m"] == p["m"]
    assert p["n2"] - c["n2"] == 581294863


def test_qkd_example_seed_length():
    # Section "Cryptomite for privacy amplification in QKD": n = 1.738e9,
    # m = 41378264, Toeplitz seed d = m + n - 1 = 1.738e9 + 41378263
    n = 1738000000
    k1 = 41378264 + 67           # 67 > 2 log2(1e10) = 66.44, so m = 41378264
    p = P.plan("toeplitz", "seeded", "quantum", n, k1, LE10)
    assert p["m"] == 41378264
    assert p["n2"] == n + 41378263


def _largest(ok, hi=1 << 40):
    lo = 0
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if ok(mid):
            lo = mid
        else:
            hi = mid
    return lo


# The base bounds, as real numbers (before the floor).
def seeded_2univ(k1, le):              # Thm. circSEED, Toeplitz theorem
    return k1 + 2 * le


def dodis_two_source(k1, k2, n, le):   # classical Dodis et al. theorem
    return k1 + k2 - n + 1 + 2 * le


def trevisan_seeded_ok(m, k1, le):     # combined-parameters theorem
    return m <= k1 + 4 * le - 4 * math.log2(m) - 6


def markov2_le0(le, m):
    # Thm. Markov2: final error sqrt(3 eps0 2^(m-2)) = eps  =>  log2 eps0
    return 2 * le - LOG3 - (m - 2)


def _cases(seed, count):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        n1 = int(rng.integers(10 ** 3, 10 ** 10))
        k1 = float(rng.uniform(0.3, 1.0) * n1)
        k2f = float(rng.uniform(0.9, 1.0))
        le = -float(rng.uniform(5, 200))
        yield n1, k1, k2f, le


def test_circulant_two_source_from_2universal_extension():
    # Thm. 2-weak-source (two-universal): seeded error eps_s becomes
    # 2^((n2-k2)/2) eps_s; with n2 = n1 + 1.  Cor. MarkovFor2Uni: same in the
    # Markov model, for either adversary.
    for n1, k1, k2f, le in _cases(1, 300):
        n2 = n1 + 1
        k2 = k2f * n2
        want = max(0, math.floor(seeded_2univ(k1, le - (n2 - k2) / 2)))
        for model in ("product", "markov"):
            for adv in ("classical", "quantum"):
                assert P.output_length("circulant", model, adv, n1, k1, le, k2=k2) == want


def test_toeplitz_two_source_from_2universal_extension():
    # the same extension with n2 = n1 + m - 1, which depends on m: the largest
    # m with m <= k1 + 2 (log2 eps - (n1 + m - 1 - k2) / 2), searched directly
    for n1, k1, k2f, le in _cases(2, 300):
        k2 = k2f * n1
        want = _largest(lambda m: m <= seeded_2univ(k1, le - (n1 + m - 1 - k2) / 2))
        for model in ("product", "markov"):
            assert P.output_length("toeplitz", model, "quantum", n1, k1, le, k2=k2) == want


def test_dodis_quantum_from_markov2():
    # Thm. Markov2 applied to the classical two-source bound: entropies lowered
    # by log2(1/eps0), eps0 from the final error; largest m searched directly
    for n1, k1, k2f, le in _cases(3, 300):
        k2 = k2f * n1

        def ok(m, k2=k2):
            le0 = markov2_le0(le, m)
            return m <= dodis_two_source(k1 + le0, k2 + le0, n1, le0)
        want = _largest(ok)
        for model in ("product", "markov"):
            assert P.output_length("dodis", model, "quantum", n1, k1, le, k2=k2) == want
        # seeded quantum: the same with a perfect seed, k2 = n
        def ok_s(m):
            le0 = markov2_le0(le, m)
            return m <= dodis_two_source(k1 + le0, n1 + le0, n1, le0)
        assert P.output_length("dodis", "seeded", "quantum", n1, k1, le) == _largest(ok_s)


def test_dodis_classical_markov_from_markov1():
    # Thm. Markov1: entropies lowered by log2(1/eps0), error 3 eps0; the
    # quantum bound also holds, and the larger one is taken
    for n1, k1, k2f, le in _cases(4, 300):
        k2 = k2f * n1
        le0 = le - LOG3
        c = max(0, math.floor(dodis_two_source(k1 + le0, k2 + le0, n1, le0)))
        q = P.output_length("dodis", "markov", "quantum", n1, k1, le, k2=k2)
        assert P.output_length("dodis", "markov", "classical", n1, k1, le, k2=k2) == max(c, q)


def test_trevisan_two_source_from_general_extension_and_markov2():
    for n1, k1, _, le in _cases(5, 120):
        d = int(np.random.default_rng(n1).integers(100, 10 ** 5))
        k2 = d * 0.995
        # Thm. 2-weak-source, general form: error 2^(n2 - k2) eps_s, n2 = d
        want = _largest(lambda m: m >= 1 and trevisan_seeded_ok(m, k1, le - (d - k2)))
        got = P.output_length("trevisan", "product", "classical", n1, k1, le, k2=k2, d=d)
        assert got == want

        # Thm. Markov2 on that two-source bound
        def okq(m):
            if m < 1:
                return True
            le0 = markov2_le0(le, m)
            return trevisan_seeded_ok(m, k1 + le0, le0 - (d - (k2 + le0)))
        assert P.output_length("trevisan", "markov", "quantum", n1, k1, le, k2=k2, d=d) == _largest(okq)


def test_two_source_with_perfect_seed_is_seeded():
    # k2 = n2 must give back the seeded bound (classical side information)
    for n1, k1, _, le in _cases(6, 200):
        Pc = oracle.next_na(n1 % 10 ** 6 + 3)
        nc = Pc - 1
        kc = min(k1, nc * 0.9)
        assert (P.output_length("circulant", "product", "classical", nc, kc, le, k2=Pc)
                == P.output_length("circulant", "seeded", "classical", nc, kc, le))
        assert (P.output_length("dodis", "product", "classical", Pc, kc, le, k2=Pc)
                == P.output_length("dodis", "seeded", "classical", Pc, kc, le))
        m = P.output_length("toeplitz", "seeded", "classical", n1, k1, le)
        if m > 0:
            assert P.output_length("toeplitz", "product", "classical", n1, k1, le,
                                   k2=n1 + m - 1) == m
        d = 10 ** 4
        assert (P.output_length("trevisan", "product", "classical", n1, k1, le, k2=d, d=d)
                == P.output_length("trevisan", "seeded", "classical", n1, k1, le))


def test_printed_overview_forms_agree():
    # the overview list prints the Dodis Markov bound with 9 - 4 log2 3 and the
    # Toeplitz two-source bound before substituting n2 = n1 + m - 1
    for n1, k1, k2f, le in _cases(7, 200):
        k2 = k2f * n1
        over = max(0, math.floor((k1 + k2 - n1 + 8 * le + 9 - 4 * LOG3) / 5))
        assert P.output_length("dodis", "markov", "quantum", n1, k1, le, k2=k2) == over
        m = P.output_length("toeplitz", "product", "quantum", n1, k1, le, k2=k2)
        if m > 0:
            assert m <= k1 + (k2 - (n1 + m - 1)) + 2 * le
            assert not (m + 1 <= k1 + (k2 - (n1 + m)) + 2 * le)


def test_trevisan_seed_length_hand_worked():
    # n1 = 2^20, m = 1000, eps = 2^-20:
    #   q = 2 ceil(20 + 2 (1 + log2 1000 + 20)) = 2 ceil(81.93) = 164
    #   t = 167 (165 = 3*5*11, 166 = 2*83, 167 prime)
    #   a = ceil((log2 994.56 - log2 161.56) / (log2 5.4366 - log2 4.4366))
    #     = ceil((9.958 - 7.336) / (2.4427 - 2.1495)) = ceil(8.94) = 9
    #   d = 9 * 167^2 = 251001
    assert P.trevisan_seed_length(2 ** 20, 1000, -20.0) == (167, 9, 251001)
    # m <= 2e: the logarithm is undefined, a = 1
    t, a, d = P.trevisan_seed_length(1000, 5, -10.0)
    assert a == 1 and d == t * t
    # t is the smallest prime >= q, by trial division
    for n1, m, le in ((10 ** 6, 10 ** 5, -30.0), (77, 3, -1.5), (2 ** 40, 2 ** 30, -100.0)):
        t, a, d = P.trevisan_seed_length(n1, m, le)
        q = 2 * math.ceil(math.log2(n1) + 2 * math.log2(2 * m) - 2 * le)
        assert t >= q and all(t % f for f in range(2, int(t ** 0.5) + 1))
        assert all(any(c % f == 0 for f in range(2, int(c ** 0.5) + 1)) for c in range(q, t))


def test_monotone_in_entropy_and_error():
    for n1, k1, k2f, le in _cases(8, 100):
        Pn = oracle.next_na(n1 % 10 ** 6 + 3)
        k = min(k1, Pn * 0.95)
        for kind in ("circulant", "dodis"):
            n = Pn - 1 if kind == "circulant" else Pn
            k = min(k, n)
            for adv in ("classical", "quantum"):
                a = P.output_length(kind, "product", adv, n, k, le, k2=0.95 * Pn)
                b = P.output_length(kind, "product", adv, n, k, le + 1, k2=0.95 * Pn)
                c = P.output_length(kind, "product", adv, n, k * 0.99, le, k2=0.95 * Pn)
                assert c <= a <= b
        # quantum never above classical for Dodis et al.
        assert (P.output_length("dodis", "seeded", "quantum", Pn, min(k, Pn), le)
                <= P.output_length("dodis", "seeded", "classical", Pn, min(k, Pn), le))


def test_plan_cut_lowers_entropy():
    # Lemma shorten-entropy: cutting c bits costs c bits of min-entropy
    n_raw = 10 ** 6
    k1 = 5e5
    down = P.plan("circulant", "seeded", "quantum", n_raw, k1, -40.0, adjust="down")
    Pd = oracle.prev_na(n_raw + 1)
    assert down["n2"] == Pd and down["cut_input"] == n_raw + 1 - Pd
    assert down["k1"] == k1 - down["cut_input"]
    up = P.plan("dodis", "product", "classical", n_raw, k1, -40.0, seed_rate=0.9, adjust="up")
    assert up["n1"] == up["n2"] == oracle.next_na(n_raw) and up["k1"] == k1
    assert up["k2"] == pytest.approx(0.9 * up["n2"])


def test_vn_expected_length_by_counting():
    # p(1-p)n: the expected count of unequal pairs (each with probability
    # 2p(1-p)) over n/2 pairs, checked by exact enumeration of n = 8
    from itertools import product
    for p in (0.5, 0.3, 0.9):
        n = 8
        exp = 0.0
        for bits in product((0, 1), repeat=n):
            pr = math.prod(p if b else 1 - p for b in bits)
            exp += pr * sum(bits[2 * j] != bits[2 * j + 1] for j in range(n // 2))
        assert P.vn_expected_length(n, p) == pytest.approx(exp)


# ----- Part 2: the C ABI against the oracle ---------------------------------

KIND = {"toeplitz": 0, "circulant": 1, "dodis": 2, "trevisan": 3}
MODEL = {"seeded": 0, "product": 1, "markov": 2}
ADV = {"classical": 0, "quantum": 1}
ADJ = {"up": 0, "down": 1, "closest": 2}


@pytest.fixture(scope="module")
def nat():
    from paper_2402_09481_gb300 import build, native
    build.build()
    native.lib()
    return native


def test_abi_output_length_matches_oracle(nat):
    rng = np.random.default_rng(11)
    primes = [oracle.next_na(int(v)) for v in rng.integers(10, 10 ** 9, 12)]
    count = 0
    for Pn in primes:
        for _ in range(6):
            le = -float(rng.uniform(1, 150))
            for kind in KIND:
                n1 = {"circulant": Pn - 1, "dodis": Pn}.get(kind, int(rng.integers(100, 10 ** 11)))
                k1 = float(rng.uniform(0.05, 1.0) * n1)
                d = int(rng.integers(50, 10 ** 6))
                seed = {"circulant": n1 + 1, "dodis": n1, "trevisan": d}.get(kind, n1)
                k2 = float(rng.uniform(0.8, 1.0) * seed)
                for model in MODEL:
                    for adv in ADV:
                        want = P.output_length(kind, model, adv, n1, k1, le, k2=k2, d=d)
                        got = nat.output_length(KIND[kind], MODEL[model], ADV[adv], n1, k1, le, k2=k2, d=d)
                        assert got == want, (kind, model, adv, n1, k1, k2, d, le)
                        count += 1
    assert count > 1000


def test_abi_plan_matches_oracle(nat):
    rng = np.random.default_rng(12)
    for _ in range(40):
        n_raw = int(rng.integers(10, 10 ** 8))
        k1 = float(rng.uniform(0.05, 1.0) * n_raw)
        le = -float(rng.uniform(1, 100))
        r = float(rng.uniform(0.9, 1.0))
        for kind in KIND:
            for model in MODEL:
                if kind == "trevisan" and model != "seeded":
                    continue
                for adv in ADV:
                    for adj in ADJ:
                        want = P.plan(kind, model, adv, n_raw, k1, le, seed_rate=r, adjust=adj)
                        got = nat.plan_params(KIND[kind], MODEL[model], ADV[adv], n_raw, k1, le,
                                              seed_rate=r, adjust=ADJ[adj])
                        for key in ("n1", "n2", "pad_input", "cut_input", "m"):
                            assert got[key] == want[key], (kind, model, adv, adj, key)
                        assert got["k1"] == pytest.approx(want["k1"], rel=1e-15)
                        assert got["k2"] == pytest.approx(want["k2"], rel=1e-15)
    # the paper's examples through the ABI
    g = nat.plan_params(0, 0, 1, 6500000000, 581295000, LE10)
    assert (g["m"], g["n2"]) == (581294933, 7081294932)
    c = nat.plan_params(1, 0, 1, 6500000000, 581295000, LE10, adjust=nat.ADJUST_CLOSEST)
    assert (c["n2"], c["pad_input"], c["m"]) == (6500000069, 68, 581294933)


def test_abi_trevisan_seed_and_closest(nat):
    assert nat.trevisan_seed_length(2 ** 20, 1000, -20.0) == (167, 9, 251001)
    rng = np.random.default_rng(13)
    for _ in range(50):
        n1, m = int(rng.integers(2, 10 ** 12)), int(rng.integers(1, 10 ** 9))
        le = -float(rng.uniform(0.5, 300))
        assert nat.trevisan_seed_length(n1, m, le) == P.trevisan_seed_length(n1, m, le)
    for n in list(range(0, 400)) + [int(v) for v in rng.integers(400, 10 ** 10, 30)]:
        assert nat.closest_na_prime(n) == oracle.closest_na(n), n
    assert nat.closest_na_prime(6500000001) == 6500000069


def test_abi_argument_checks(nat):
    E = nat.CM_EINVAL
    bad = [
        (0, 0, 0, 100, 50.0, 0.0),        # log2 eps = 0
        (0, 0, 0, 100, 50.0, float("nan")),
        (0, 0, 0, 100, 150.0, -10.0),     # k1 > n1
        (0, 0, 0, 100, -1.0, -10.0),
        (0, 0, 0, 0, 0.0, -10.0),         # n1 = 0
        (1, 0, 0, 6, 5.0, -10.0),         # 7 is prime but 2 is not a primitive root
        (2, 0, 0, 100, 50.0, -10.0),      # Dodis et al. n1 not prime
        (4, 0, 0, 100, 50.0, -10.0),      # unknown kind
        (0, 3, 0, 100, 50.0, -10.0),      # unknown model
        (0, 0, 2, 100, 50.0, -10.0),      # unknown adversary
    ]
    for kind, model, adv, n1, k1, le in bad:
        with pytest.raises(nat.CMError) as e:
            nat.output_length(kind, model, adv, n1, k1, le)
        assert e.value.status == E
    with pytest.raises(nat.CMError):
        nat.output_length(1, 1, 0, 106, 50.0, -10.0, k2=200.0)       # k2 above the 107-bit seed
    with pytest.raises(nat.CMError):
        nat.output_length(3, 1, 0, 1000, 500.0, -10.0, k2=10.0, d=0)  # Trevisan two-source needs d
    with pytest.raises(nat.CMError):
        nat.plan_params(3, 1, 0, 1000, 500.0, -10.0, seed_rate=0.9)   # Trevisan plan is seeded only
    with pytest.raises(nat.CMError):
        nat.plan_params(1, 1, 0, 1000, 500.0, -10.0, seed_rate=1.5)
    with pytest.raises(nat.CMError):
        nat.plan_params(1, 0, 0, 1, 1.0, -10.0, adjust=nat.ADJUST_DOWN)  # no N_A member <= 2
    with pytest.raises(nat.CMError):
        nat.trevisan_seed_length(10, 0, -5.0)
    # nothing extractable: m = 0, not an error
    assert nat.output_length(0, 0, 0, 100, 10.0, -10.0) == 0
