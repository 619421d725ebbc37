"""Blocked extractions (products split over input blocks and output windows)
against the oracle.

A context whose transform limit is lowered (cm_options.max_transform_lg = 8 ..
19) splits ordinary sizes into many input blocks and output windows, so every
block path (single-CTA blocks XORed, one-pass and two-pass blocks summed in
the transform domain, sum groups capped by max_sum_blocks and XORed, the
Circulant pad bit in the block that holds it, a short last input block padded
to the window's common length, the double wrap of the seed index, output
windows that end mid-word, the Dodis et al. precondition) is compared bit for
bit with the oracle's whole output, over both fields.  At the default limit
the planner splits by cost alone (shorter products and a dense tail of the
terms that do not fit, instead of one 2^23 transform; the Circulant
workload as two summed 2^24 products and an 83-term tail, checked against the
single 2^25 transform bit for bit;
Dodis et al. at n = 2^30 as two 2^30 products over the 32-bit field), and the
QRNG example's sizes (n = 6.5e9, m = 581294933, Section "Cryptomite for
randomness extraction in (Q)RNG") run as 14 summed products of 2^30 in three
sum groups; those and the one-transform extreme L = 2^32 are compared on
sampled rows.
"""

import numpy as np
import pytest
import torch

import oracle
from oracle import extractors as ex
from paper_2402_09481_gb300 import inputs, native
from conftest import from_dev, to_dev

pytestmark = pytest.mark.gpu
T, C, D = native.TOEPLITZ, native.CIRCULANT, native.DODIS


@pytest.fixture(scope="module")
def ctxs():
    from paper_2402_09481_gb300 import build
    build.build()
    cs = {lg: native.Context(0, max_transform_lg=lg) for lg in (8, 12, 14, 15, 16, 18, 19)}
    cs["14s2"] = native.Context(0, max_transform_lg=14, max_sum_blocks=2)
    cs["16s3"] = native.Context(0, max_transform_lg=16, max_sum_blocks=3)
    cs["15gl"] = native.Context(0, max_transform_lg=15, field=native.FIELD_GOLDILOCKS)
    cs["17gls2"] = native.Context(0, max_transform_lg=17, field=native.FIELD_GOLDILOCKS, max_sum_blocks=2)
    cs["16gl"] = native.Context(0, max_transform_lg=16, field=native.FIELD_GOLDILOCKS)
    yield cs
    for c in cs.values():
        c.close()


def run(ctx, kind, n, m, xw, yw):
    x, y = to_dev(xw), to_dev(yw)
    z = torch.full((native.words(m),), -1, dtype=torch.int64, device="cuda")
    if kind == T:
        ctx.toeplitz(x, n, y, m, z)
    elif kind == C:
        ctx.circulant(x, n, y, m, z)
    else:
        ctx.dodis(x, y, n, m, z)
    torch.cuda.synchronize()
    return from_dev(z)


def want(kind, n, m, xw, yw):
    if kind == T:
        return oracle.toeplitz_packed(xw, n, yw, m)
    if kind == C:
        return oracle.circulant_packed(xw, n, yw, m)
    return oracle.dodis_packed(xw, yw, n, m)


def ybits(kind, n, m):
    return n + m - 1 if kind == T else (n + 1 if kind == C else n)


CASES = [
    # (kind, n, m, max_transform_lg)
    (T, 1000, 300, 8), (T, 777, 129, 8), (T, 5000, 2000, 12), (T, 20000, 3000, 12),
    (T, 100000, 30000, 15), (T, 300000, 1000, 14), (T, 70000, 70000, 16), (T, 4097, 4096, 12),
    (T, 400_003, 131_077, 19),
    (C, "P5000", 0.5, 12), (C, "P5000", 0.1, 8), (C, "P200000", 0.5, 16), (C, "P200000", 0.05, 14),
    (C, "P300000", 0.3, 18),
    (D, "P50000", 0.4, 14), (D, "P3000", 0.9, 8), (D, "P300000", 0.2, 16),
    # sum groups of at most 2 or 3 products, XORed; Goldilocks sums
    (T, 100000, 3000, "14s2"), (T, 300000, 20000, "16s3"), (C, "P200000", 0.1, "14s2"),
    (D, "P300000", 0.3, "16s3"), (T, 100000, 30000, "15gl"), (C, "P300000", 0.2, "17gls2"),
    (D, "P100000", 0.5, "15gl"),
]


def limit(lg):
    return lg if isinstance(lg, int) else int(lg[:2])


def resolve(kind, n, m):
    if isinstance(n, str):
        P = oracle.next_na(int(n[1:]))
        n = P - 1 if kind == C else P
        m = max(1, int(m * n))
    return n, m


@pytest.mark.parametrize("kind,n,m,lg", CASES)
def test_blocked_matches_oracle(ctxs, cm_ctx, kind, n, m, lg):
    n, m = resolve(kind, n, m)
    assert native.block_count(kind, n, m, limit(lg)) > 1
    xw = inputs.bernoulli_half(900 + n % 97, n)
    if kind == D:
        xw[0] = (xw[0] | np.uint64(1)) & ~np.uint64(2)
    yw = inputs.bernoulli_half(901 + n % 89, ybits(kind, n, m))
    got = run(ctxs[lg], kind, n, m, xw, yw)
    assert (got == want(kind, n, m, xw, yw)).all(), (kind, n, m, lg)
    # the same bits as the one-transform call
    assert (got == run(cm_ctx, kind, n, m, xw, yw)).all()


def test_blocked_dodis_precondition(ctxs):
    P = oracle.next_na(20000)
    for fill in (0, 1):
        xw = ex.pack_bits(np.full(P, fill, dtype=np.uint8))
        yw = inputs.bernoulli_half(5, P)
        got = run(ctxs[12], D, P, P // 2, xw, yw)
        assert not got.any()
        assert ctxs[12].device_status()[0] == native.CM_EPRECOND


def test_blocked_host_buffers(ctxs):
    n, m = 50000, 9000
    xw, yw = inputs.bernoulli_half(11, n), inputs.bernoulli_half(12, n + m - 1)
    xh = torch.from_numpy(xw.view(np.int64))
    yh = torch.from_numpy(yw.view(np.int64))
    zh = torch.zeros(native.words(m), dtype=torch.int64)
    assert ctxs[12].extract_host(T, xh, n, yh, m, zh) == native.CM_OK
    assert (zh.numpy().view(np.uint64) == oracle.toeplitz_packed(xw, n, yw, m)).all()


def sample_rows(m, k, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([np.arange(16), np.arange(m - 16, m), rng.integers(0, m, k)]))


def out_bits(z, rows):
    return ((z[rows >> 6] >> (rows & 63).astype(np.uint64)) & np.uint64(1)).astype(np.uint8)


TAIL_CASES = [
    # (kind, n, m, context): products of 2^14 .. 2^16 plus a dense tail of
    # 136, 71, 202, 200 terms (one product; two summed; one; two windows)
    (C, 16_420, 100, 14), (C, 16_420, 8_210, 14), (D, 32_771, 200, 15), (T, 35_721, 60_000, 16),
    (T, 35_721, 60_000, "16gl"),
]


@pytest.mark.parametrize("kind,n,m,lg", TAIL_CASES)
def test_dense_tail_matches_oracle(ctxs, kind, n, m, lg):
    info = native.plan_query(kind, n, m, max_transform_lg=limit(lg),
                             field=native.FIELD_GOLDILOCKS if str(lg).endswith("gl") else native.FIELD_AUTO)
    assert info["tail_terms"] > 0
    xw = inputs.bernoulli_half(70 + n % 13, n)
    if kind == D:
        xw[0] = (xw[0] | np.uint64(1)) & ~np.uint64(2)
    yw = inputs.bernoulli_half(71 + n % 11, ybits(kind, n, m))
    assert (run(ctxs[lg], kind, n, m, xw, yw) == want(kind, n, m, xw, yw)).all()


def test_dense_tail_dodis_precondition(ctxs):
    # a constant source zeroes the output of a plan with a tail as well
    P = 32_771
    for fill in (0, 1):
        xw = ex.pack_bits(np.full(P, fill, dtype=np.uint8))
        got = run(ctxs[15], D, P, 200, xw, inputs.bernoulli_half(74, P))
        assert not got.any()
        assert ctxs[15].device_status()[0] == native.CM_EPRECOND


FOLD_CASES = [
    # (kind, n, m): two summed 2^14 products and a dense tail in one window:
    # the tail runs inside the window's pack (71 and 241 terms)
    (C, 16_420, 8_210),
    (D, 17_011, 8_000),
]


@pytest.mark.parametrize("kind,n,m", FOLD_CASES)
def test_tail_folded_into_pack(kind, n, m):
    ctx = native.Context(0, max_transform_lg=14)
    try:
        info = native.plan_query(kind, n, m, max_transform_lg=14)
        assert info["products"] == 2 and info["windows"] == 1 and info["tail_terms"] > 0
        xw = inputs.bernoulli_half(80 + n % 7, n)
        if kind == D:
            xw[0] = (xw[0] | np.uint64(1)) & ~np.uint64(2)
        yw = inputs.bernoulli_half(81 + n % 5, ybits(kind, n, m))
        ctx.profile_enable(True)
        ctx.profile_read(reset=True)
        z = run(ctx, kind, n, m, xw, yw)
        prof = ctx.profile_read(reset=True)
        ctx.profile_enable(False)
        assert "k_pack_tail" in prof and "k_tail" not in prof and "k_pack" not in prof, prof
        assert sum(c for c, _ in prof.values()) == info["launches"]
        assert (z == want(kind, n, m, xw, yw)).all()
        if kind == D:  # a constant source still zeroes the output
            for fill in (0, 1):
                got = run(ctx, D, n, m, ex.pack_bits(np.full(n, fill, dtype=np.uint8)), yw)
                assert not got.any()
                assert ctx.device_status()[0] == native.CM_EPRECOND
    finally:
        ctx.close()


FUSED_CASES = [
    # (kind, n, m, max_transform_lg, max_sum_blocks): products of 2^22 .. 2^25
    # over q = 5 * 2^25 + 1 run the fused column passes (tiles of 2^9 .. 2^12
    # rows); alone, summed in pairs, and in groups of three (inner sums)
    (T, 2 ** 21, 2 ** 21, 22, 0),
    (T, 3 * 2 ** 21 + 5, 2 ** 21 - 7, 23, 0),
    (T, 2 ** 24 - 1000, 12_345, 24, 0),
    (T, 9_000_001, 777_777, 22, 0),
    (C, "P9000000", 0.3, 23, 3),
    (D, "P12000000", 0.4, 24, 2),
]


@pytest.mark.parametrize("kind,n,m,lg,sums", FUSED_CASES)
def test_fused_passes_sampled(kind, n, m, lg, sums):
    n, m = resolve(kind, n, m)
    ctx = native.Context(0, max_transform_lg=lg, max_sum_blocks=sums)
    q30 = native.Context(0, max_transform_lg=lg, max_sum_blocks=sums, field=native.FIELD_Q30)
    try:
        xw = inputs.bernoulli_half(930 + n % 61, n)
        if kind == D:
            xw[0] = (xw[0] | np.uint64(1)) & ~np.uint64(2)
        yw = inputs.bernoulli_half(931 + n % 59, ybits(kind, n, m))
        z = run(ctx, kind, n, m, xw, yw)
        # every bit equals the other field's kernels; sampled rows the oracle's
        assert (z == run(q30, kind, n, m, xw, yw)).all()
        rows = sample_rows(m, 48, 7)
        rowf = {T: lambda: oracle.toeplitz_rows(xw, n, yw, m, rows),
                C: lambda: oracle.circulant_rows(xw, n, yw, m, rows),
                D: lambda: oracle.dodis_rows(xw, yw, n, m, rows)}[kind]
        assert (out_bits(z, rows) == rowf()).all()
        if m & 63:
            assert int(z[-1]) >> (m & 63) == 0
    finally:
        ctx.close()
        q30.close()


def test_split_by_cost(cm_ctx):
    # K + m - 1 = 2^22 + 149: shorter products and a dense tail instead of one
    # 2^23 transform
    n, m = 2 ** 22 + 50, 100
    info = native.plan_query(T, n, m)
    assert info["transform_length"] <= 2 ** 22 and info["tail_terms"] > 0
    xw, yw = inputs.bernoulli_half(66, n), inputs.bernoulli_half(67, n + m - 1)
    assert (run(cm_ctx, T, n, m, xw, yw) == oracle.toeplitz_packed(xw, n, yw, m)).all()


def test_circulant_workload_plans_agree(cm_ctx):
    # n + 1 = 16777259, m = n / 2: two summed 2^24 products and an 83-term
    # tail; every output bit equals the single 2^25 transform's
    n = 16777258
    m = n // 2
    assert native.plan_query(C, n, m)["tail_terms"] == 83
    xw, yw = inputs.bernoulli_half(72, n), inputs.bernoulli_half(73, n + 1)
    z = run(cm_ctx, C, n, m, xw, yw)
    single = native.Context(0, plan_mode=native.PLAN_SINGLE)
    try:
        assert (run(single, C, n, m, xw, yw) == z).all()
    finally:
        single.close()
    rows = sample_rows(m, 64, 5)
    assert (out_bits(z, rows) == oracle.circulant_rows(xw, n, yw, m, rows)).all()


@pytest.mark.slow
def test_dodis_workload_both_plans(cm_ctx):
    # n = 2^30 - 35, m = 0.4 n: two 2^30 products over the 32-bit field, and
    # one Goldilocks transform of 2^31 (single mode): same bits
    n = 1073741789
    m = int(0.4 * n)
    assert native.plan_query(D, n, m)["products"] == 2
    xw, yw = inputs.bernoulli_half(68, n), inputs.bernoulli_half(69, n)
    z = run(cm_ctx, D, n, m, xw, yw)
    rows = sample_rows(m, 16, 4)
    assert (out_bits(z, rows) == oracle.dodis_rows(xw, yw, n, m, rows)).all()
    single = native.Context(0, field=native.FIELD_GOLDILOCKS, plan_mode=native.PLAN_SINGLE)
    try:
        assert (run(single, D, n, m, xw, yw) == z).all()
    finally:
        single.close()


@pytest.mark.slow
def test_dodis_workload_biased_source(cm_ctx):
    # the configuration's second Dodis et al. run: x 0.8-biased (P(bit = 1) =
    # 0.8), y Bernoulli(1/2), n = 2^30 - 35, m = floor(0.4 n); sampled rows
    n = 1073741789
    m = int(0.4 * n)
    xw, yw = inputs.bernoulli(70, n), inputs.bernoulli_half(71, n)
    z = run(cm_ctx, D, n, m, xw, yw)
    assert cm_ctx.device_status()[0] == native.CM_OK
    rows = sample_rows(m, 16, 8)
    assert (out_bits(z, rows) == oracle.dodis_rows(xw, yw, n, m, rows)).all()
    if m & 63:
        assert int(z[-1]) >> (m & 63) == 0


@pytest.mark.slow
def test_qrng_example_toeplitz_sampled(cm_ctx):
    # n1 = 6.5e9, m = floor(k1 + 2 log2 1e-10) = 581294933, seed n1 + m - 1 bits
    n, m = 6_500_000_000, 581_294_933
    assert native.block_count(T, n, m) == 14
    xw, yw = inputs.bernoulli_half(60, n), inputs.bernoulli_half(61, n + m - 1)
    z = run(cm_ctx, T, n, m, xw, yw)
    rows = sample_rows(m, 24, 1)
    assert (out_bits(z, rows) == oracle.toeplitz_rows(xw, n, yw, m, rows)).all()
    if m & 63:
        assert int(z[-1]) >> (m & 63) == 0


@pytest.mark.slow
def test_qkd_example_toeplitz_sampled(cm_ctx):
    # Section "Cryptomite for privacy amplification in QKD": n = 1.738e9 raw
    # key bits, m = 41378264, seed n + m - 1 bits
    n, m = 1_738_000_000, 41_378_264
    xw, yw = inputs.bernoulli_half(64, n), inputs.bernoulli_half(65, n + m - 1)
    z = run(cm_ctx, T, n, m, xw, yw)
    rows = sample_rows(m, 24, 6)
    assert (out_bits(z, rows) == oracle.toeplitz_rows(xw, n, yw, m, rows)).all()
    if m & 63:
        assert int(z[-1]) >> (m & 63) == 0


@pytest.mark.slow
def test_qrng_example_circulant_sampled(cm_ctx):
    # the Circulant extension of the same example: P = 6.5e9 + 69, n1' = P - 1
    n, m = 6_500_000_068, 581_294_933
    assert oracle.is_prime(n + 1) and native.block_count(C, n, m) == 14
    xw, yw = inputs.bernoulli_half(62, n), inputs.bernoulli_half(63, n + 1)
    z = run(cm_ctx, C, n, m, xw, yw)
    rows = sample_rows(m, 16, 2)
    assert (out_bits(z, rows) == oracle.circulant_rows(xw, n, yw, m, rows)).all()


@pytest.mark.slow
def test_one_transform_of_length_2_32(cm_ctx):
    n, m = 2 ** 31, 2 ** 31 + 1
    assert native.ntt_length(T, n, m) == 2 ** 32 and native.block_count(T, n, m) == 1
    xw, yw = inputs.bernoulli_half(64, n), inputs.bernoulli_half(65, n + m - 1)
    z = run(cm_ctx, T, n, m, xw, yw)
    rows = sample_rows(m, 16, 3)
    assert (out_bits(z, rows) == oracle.toeplitz_rows(xw, n, yw, m, rows)).all()
