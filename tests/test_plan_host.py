"""The block planner's product lists, checked on the CPU.

cm_plan_products lists the middle products one call runs: their bit maps over x
and y, transform lengths, output windows and how their transform-domain
products are summed (sum groups) or XORed.  These tests need no GPU:

- structure: windows tile [0, m) in order, input blocks tile the K terms, the
  products of a sum group share K, m and L, the window fits its transform, and
  no group can hold a count at or above its 32-bit field's prime (3 * 2^30 + 1
  or 5 * 2^25 + 1);
- value: the listed products, evaluated exactly in numpy (maps as the header
  defines them, cyclic convolution of length L, window K - 1 .. K + m - 2,
  sums taken modulo the product's field, parity, XOR) give the oracle's
  output bit for bit, for forced and cost-chosen splits of all three
  extractors.
"""

import numpy as np
import pytest

import oracle
from oracle import extractors as ex
from paper_2402_09481_gb300 import inputs, native

T, C, D = native.TOEPLITZ, native.CIRCULANT, native.DODIS
Q30 = 3 * 2 ** 30 + 1
Q25 = 5 * 2 ** 25 + 1
PRIME = {native.FIELD_Q30: Q30, native.FIELD_Q25: Q25}


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2402_09481_gb300 import build
    build.build()


def k_terms(kind, n):
    return n + 1 if kind == C else n


def ybits(kind, n, m):
    return n + m - 1 if kind == T else (n + 1 if kind == C else n)


def map_bits(src, mode, length, srclen, off, L):
    """Values of a product's bit map at transform positions 0 .. L - 1."""
    k = np.arange(L, dtype=np.int64)
    ok = k < length
    if mode == 0:
        idx = k
    elif mode == 1:
        idx = (k + off) % srclen
    else:
        idx = off - k
        ok &= (idx >= 0) & (idx < srclen)
    v = np.zeros(L, dtype=np.int64)
    v[ok] = src[idx[ok]]
    return v


def cyclic_conv(a, b):
    """Exact cyclic convolution of two 0/1 vectors (counts <= L < 2^24)."""
    L = a.size
    c = np.fft.irfft(np.fft.rfft(a.astype(np.float64)) * np.fft.rfft(b.astype(np.float64)), L)
    r = np.rint(c)
    assert np.abs(c - r).max() < 0.25
    return r.astype(np.int64)


def emulate(kind, n, m, xw, yw, prods):
    xb = ex.unpack_bits(xw, n)
    yb = ex.unpack_bits(yw, ybits(kind, n, m))
    z = np.zeros(m, dtype=np.uint8)
    acc = None
    for p in prods:
        if p["sum"] == 4:  # dense tail over the whole product's maps
            T, K = p["tail_terms"], p["K"]
            a = map_bits(xb, p["a_mode"], p["a_len"], p["a_srclen"], p["a_off"], K)
            b = map_bits(yb, p["b_mode"], p["b_len"], p["b_srclen"], p["b_off"], m + T)
            tail = np.zeros(m, dtype=np.int64)
            for t in range(T):
                if a[K - 1 - t]:
                    tail += b[t:t + m]
            z ^= (tail & 1).astype(np.uint8)
            continue
        L, K, mr = p["L"], p["K"], p["m"]
        a = map_bits(xb, p["a_mode"], p["a_len"], p["a_srclen"], p["a_off"], L)
        b = map_bits(yb, p["b_mode"], p["b_len"], p["b_srclen"], p["b_off"], L)
        win = cyclic_conv(a, b)[K - 1:K - 1 + mr]
        acc = win.copy() if p["sum"] in (0, 1) else acc + win
        if p["sum"] in (0, 3):
            # Goldilocks: every count (< 2^40) is below the prime, nothing wraps
            s = acc % PRIME[p["field"]] if p["field"] in PRIME else acc
            par = (s & 1).astype(np.uint8)
            lo = p["zword"] * 64
            if p["xor_into"]:
                z[lo:lo + mr] ^= par
            else:
                z[lo:lo + mr] = par
    return ex.pack_bits(z)


def want(kind, n, m, xw, yw):
    if kind == T:
        return oracle.toeplitz_packed(xw, n, yw, m)
    if kind == C:
        return oracle.circulant_packed(xw, n, yw, m)
    return oracle.dodis_packed(xw, yw, n, m)


def check_structure(kind, n, m, prods):
    K = k_terms(kind, n)
    if prods and prods[-1]["sum"] == 4:
        tail = prods[-1]
        assert 0 < tail["tail_terms"] <= 256 and tail["L"] == 0 and tail["K"] == K and tail["m"] == m
        K -= tail["tail_terms"]
        prods = prods[:-1]
    assert all(p["sum"] != 4 for p in prods)
    i = 0
    next_word = 0
    while i < len(prods):
        zw = prods[i]["zword"]
        assert zw == next_word
        win = [p for p in prods[i:] if p["zword"] == zw]
        i += len(win)
        mr = win[0]["m"]
        assert all(p["m"] == mr for p in win)
        # input blocks tile the K terms (a short block is zero past a_len)
        assert sum(p["a_len"] for p in win) == K
        # sum groups: 1, 2 .., 3 or a lone 0; members share K and L
        j = 0
        first_group = True
        while j < len(win):
            p = win[j]
            if p["sum"] == 0:
                grp = [p]
            else:
                assert p["sum"] == 1
                k = j + 1
                while win[k]["sum"] == 2:
                    k += 1
                assert win[k]["sum"] == 3
                grp = win[j:k + 1]
            assert len({(g["K"], g["L"], g["field"]) for g in grp}) == 1
            g0 = grp[0]
            assert g0["K"] - 1 + mr <= g0["L"]
            if g0["field"] == native.FIELD_Q30:
                assert g0["L"] <= 2 ** 30 and len(grp) * g0["K"] < Q30
            if g0["field"] == native.FIELD_Q25:
                assert g0["L"] <= 2 ** 25 and len(grp) * g0["K"] < Q25
            assert grp[-1]["xor_into"] == (0 if first_group else 1)
            assert all(g["xor_into"] == 0 for g in grp[:-1])
            first_group = False
            j += len(grp)
        next_word = zw + (mr + 63) // 64
        if i < len(prods):
            assert mr % 64 == 0  # windows other than the last end on a word
    assert (next_word - 1) * 64 < m <= next_word * 64


CASES = [
    # (kind, n, m, options)
    (T, 100_000, 3_000, dict(max_transform_lg=14, max_sum_blocks=2)),
    (T, 100_000, 3_000, dict(max_transform_lg=14)),
    (T, 40_000, 20_000, dict(max_transform_lg=14)),
    (T, 30_000, 70_000, dict(max_transform_lg=15, max_sum_blocks=3)),
    (T, 20_000, 3_000, dict(max_transform_lg=12)),
    (T, 1_000, 300, dict(max_transform_lg=8)),
    (T, 50_000, 9_000, dict(max_transform_lg=14, field=native.FIELD_GOLDILOCKS)),
    (T, 2 ** 22 + 50, 100, {}),  # products of 2^21 or 2^22 and a dense tail, not one 2^23
    (T, 2 ** 22 + 50, 100, dict(max_transform_lg=21)),  # three 2^21 products
    # dense tails: one product and 136 / 202 tail terms, two summed products
    # and 71, two output windows sharing a 200-term tail, over both fields
    (C, 16_420, 100, dict(max_transform_lg=14)),
    (C, 16_420, 8_210, dict(max_transform_lg=14)),
    (D, 32_771, 200, dict(max_transform_lg=15)),
    (T, 35_721, 60_000, dict(max_transform_lg=16)),
    (T, 35_721, 60_000, dict(max_transform_lg=16, field=native.FIELD_GOLDILOCKS)),
    (D, 32_771, 13_108, dict(max_transform_lg=15, field=native.FIELD_GOLDILOCKS)),
    (C, "P60000", 0.5, dict(max_transform_lg=14)),
    (C, "P60000", 0.05, dict(max_transform_lg=14, max_sum_blocks=2)),
    (C, "P5000", 0.5, dict(max_transform_lg=12)),
    (D, "P30000", 0.4, dict(max_transform_lg=14, max_sum_blocks=3)),
    (D, "P3000", 0.9, dict(max_transform_lg=8)),
]


def resolve(kind, n, m):
    if isinstance(n, str):
        P = oracle.next_na(int(n[1:]))
        n = P - 1 if kind == C else P
        m = max(1, int(m * n))
    return n, m


@pytest.mark.parametrize("kind,n,m,opts", CASES)
def test_products_reproduce_oracle(kind, n, m, opts):
    n, m = resolve(kind, n, m)
    prods = native.plan_products(kind, n, m, **opts)
    assert len(prods) > 1
    check_structure(kind, n, m, prods)
    xw = inputs.bernoulli_half(700 + n % 91, n)
    if kind == D:
        xw[0] = (xw[0] | np.uint64(1)) & ~np.uint64(2)
    yw = inputs.bernoulli_half(701 + n % 83, ybits(kind, n, m))
    assert (emulate(kind, n, m, xw, yw, prods) == want(kind, n, m, xw, yw)).all()


@pytest.mark.parametrize("kind,n,m", [
    (T, 6_500_000_000, 581_294_933), (C, 6_500_000_068, 581_294_933), (D, 1_073_741_789, 429_496_715),
    (T, 2 ** 40, 5), (T, 5, 2 ** 40), (T, 2 ** 35, 2 ** 33), (C, 16_777_258, 8_388_629), (T, 2 ** 16, 2 ** 15),
    (T, 2 ** 31, 2 ** 31 + 1),
])
def test_structure_at_large_sizes(kind, n, m):
    prods = native.plan_products(kind, n, m)
    check_structure(kind, n, m, prods)
    info = native.plan_query(kind, n, m)
    tail = [p for p in prods if p["sum"] == 4]
    prods = [p for p in prods if p["sum"] != 4]
    assert info["products"] == len(prods)
    assert info["tail_terms"] == (tail[0]["tail_terms"] if tail else 0)
    assert info["transform_length"] == max(p["L"] for p in prods)
    assert info["windows"] == len({p["zword"] for p in prods})


def test_planner_choices():
    # one transform where it is cheapest: the Circulant and Toeplitz workloads
    assert native.plan_query(T, 2 ** 16, 2 ** 15)["products"] == 1
    # the Circulant workload (n + 1 = 2^24 + 43, m = n / 2): two summed 2^24
    # products and an 83-term dense tail instead of one 2^25 transform
    c = native.plan_query(C, 16_777_258, 8_388_629)
    assert (c["products"], c["transform_length"], c["tail_terms"]) == (2, 2 ** 24, 83)
    assert native.plan_query(C, 16_777_258, 8_388_629, plan_mode=native.PLAN_SINGLE)["transform_length"] == 2 ** 25
    # Dodis et al. at n = 2^30: two summed 2^30 products over the 32-bit field
    # instead of one Goldilocks transform of 2^31; forced Goldilocks keeps 2^31
    d = native.plan_query(D, 1_073_741_789, 429_496_715)
    assert (d["products"], d["windows"], d["field"], d["transform_length"]) == (2, 1, native.FIELD_Q30, 2 ** 30)
    g = native.plan_query(D, 1_073_741_789, 429_496_715, field=native.FIELD_GOLDILOCKS,
                          plan_mode=native.PLAN_SINGLE)
    assert (g["products"], g["transform_length"], g["field"]) == (1, 2 ** 31, native.FIELD_GOLDILOCKS)
    assert d["est_ms"] < g["est_ms"] / 2
    # Goldilocks alone still prefers two summed 2^30 products (one inverse)
    g2 = native.plan_query(D, 1_073_741_789, 429_496_715, field=native.FIELD_GOLDILOCKS)
    assert (g2["products"], g2["transform_length"]) == (2, 2 ** 30) and g2["est_ms"] < g["est_ms"]
    # single mode splits only what one transform cannot hold
    assert native.plan_query(T, 6_500_000_000, 581_294_933, plan_mode=native.PLAN_SINGLE)["products"] == 14
    # the QRNG example: 14 products of 2^30 in one window, summed in groups
    # that keep every count below 3 * 2^30 + 1
    prods = native.plan_products(T, 6_500_000_000, 581_294_933)
    assert len(prods) == 14 and {p["L"] for p in prods} == {2 ** 30}
    assert [p["sum"] for p in prods].count(3) == 3
    # a budget that cannot hold the three 2^30 buffers of a summed product
    # pushes the planner to smaller products
    small = native.plan_query(T, 6_500_000_000, 581_294_933, hbm_budget_bytes=8 << 30)
    assert small["scratch_bytes"] <= 8 << 30 and small["transform_length"] < 2 ** 30


def test_plan_query_rejects():
    with pytest.raises(native.CMError):
        native.plan_query(T, 100, 50, max_transform_lg=7)
    with pytest.raises(native.CMError):
        native.plan_query(T, 100, 50, field=3)
    with pytest.raises(native.CMError):
        native.plan_query(T, 100, 50, plan_mode=2)
    with pytest.raises(native.CMError):
        native.plan_query(T, 2 ** 40, 2 ** 40)  # more than 65536 products
    with pytest.raises(native.CMError):
        native.plan_query(C, 6, 3)  # 7 is not in N_A


def random_cases(count, seed=2402):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        kind = int(rng.integers(0, 3))
        n = int(rng.integers(200, 60_000))
        if kind == C:
            n = oracle.next_na(n + 1) - 1
        elif kind == D:
            n = oracle.next_na(n)
        m = int(rng.integers(1, (20_000 if kind == T else n) + 1))
        opts = dict(max_transform_lg=int(rng.choice([8, 10, 12, 14, 15, 16])),
                    max_sum_blocks=int(rng.choice([0, 2, 3])),
                    field=int(rng.choice([native.FIELD_AUTO, native.FIELD_GOLDILOCKS, native.FIELD_Q30])))
        try:
            prods = native.plan_products(kind, n, m, **opts)
        except native.CMError:  # more than 65536 products at the smallest limits
            continue
        if len(prods) > 1:
            out.append((kind, n, m, opts))
    return out


@pytest.mark.parametrize("kind,n,m,opts", random_cases(24))
def test_random_plans_reproduce_oracle(kind, n, m, opts):
    # seeded random lengths, limits, sum caps and fields: every listed product
    # list reproduces the oracle's output bit for bit
    prods = native.plan_products(kind, n, m, **opts)
    check_structure(kind, n, m, prods)
    xw = inputs.bernoulli_half(800 + n % 71, n)
    if kind == D:
        xw[0] = (xw[0] | np.uint64(1)) & ~np.uint64(2)
    yw = inputs.bernoulli_half(801 + m % 67, ybits(kind, n, m))
    assert (emulate(kind, n, m, xw, yw, prods) == want(kind, n, m, xw, yw)).all()
