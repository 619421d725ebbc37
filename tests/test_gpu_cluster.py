"""The one-launch cluster path (transform lengths 2^14 .. 2^17 over the field
5 * 2^25 + 1: one thread-block cluster of L / 2^13 CTAs, operands in
distributed shared memory) against the oracle, bit for bit: every length, all
three extractors, ragged and maximal m, K + m - 1 equal to L, the Toeplitz
2^16 configuration; and the trace shows that the single launch ran."""

import numpy as np
import pytest

import oracle
from paper_2402_09481_gb300 import inputs, native
from conftest import from_dev, to_dev

pytestmark = pytest.mark.gpu
T, C, D = native.TOEPLITZ, native.CIRCULANT, native.DODIS


def ybits(kind, n, m):
    return n + m - 1 if kind == T else (n + 1 if kind == C else n)


def run(ctx, kind, n, m, seed):
    xw = inputs.bernoulli_half(seed, n)
    yw = inputs.bernoulli_half(seed + 1, ybits(kind, n, m))
    if kind == D:
        xw[0] = (xw[0] | np.uint64(1)) & ~np.uint64(2)
    x, y = to_dev(xw), to_dev(yw)
    ctx.profile_enable(True)
    ctx.profile_read(reset=True)
    if kind == T:
        z = ctx.toeplitz(x, n, y, m)
    elif kind == C:
        z = ctx.circulant(x, n, y, m)
    else:
        z = ctx.dodis(x, y, n, m)
    prof = ctx.profile_read(reset=True)
    ctx.profile_enable(False)
    return xw, yw, from_dev(z), prof


def want(kind, xw, n, yw, m):
    if kind == T:
        return oracle.toeplitz_packed(xw, n, yw, m)
    if kind == C:
        return oracle.circulant_packed(xw, n, yw, m)
    return oracle.dodis_packed(xw, yw, n, m)


def na(v):
    return oracle.next_na(v)


# (kind, n, m): K + m - 1 in (2^13, 2^17]
CASES = [
    (T, 2 ** 16, 2 ** 15),                # the Toeplitz 2^16 configuration (L = 2^17)
    (T, 100000, 31073),                   # K + m - 1 = 2^17 exactly
    (T, 65537, 65536),                    # K + m - 1 = 2^17 exactly, m = 2^16
    (T, 8193, 1),                         # L = 2^14, m = 1
    (T, 9000, 7000),                      # L = 2^14, ragged
    (T, 2 ** 14, 2 ** 14 + 1),            # K + m - 1 = 2^15 exactly
    (T, 20000, 12000),                    # L = 2^15
    (T, 33333, 22222),                    # L = 2^16, ragged
    (T, 1, 2 ** 15),                      # n = 1: z = y shifted
    (C, na(9000) - 1, na(9000) - 1),      # maximal m (m = n)
    (C, na(40000) - 1, 20000),            # L = 2^16
    (C, na(60000) - 1, 12345),            # L = 2^17
    (D, na(10000), na(10000)),            # maximal m
    (D, na(30000), 12000),                # L = 2^16
    (D, na(70000), 40001),                # L = 2^17 (sampled beside the full check below)
]


@pytest.mark.parametrize("kind,n,m", CASES)
def test_cluster_path_matches_oracle(cm_ctx, kind, n, m):
    info = native.plan_query(kind, n, m)
    assert 2 ** 14 <= info["transform_length"] <= 2 ** 17 and info["products"] == 1
    xw, yw, z, prof = run(cm_ctx, kind, n, m, 7000 + n % 1000 + m % 77)
    assert "k_cluster_f25" in prof and prof["k_cluster_f25"][0] == 1, prof
    assert not any(k.startswith(("k_middle", "k_pass", "k_pack")) for k in prof), prof
    assert info["launches"] == (2 if kind == D else 1)
    if m & 63:
        assert int(z[-1]) >> (m & 63) == 0
    if m <= 40000:
        assert (z == want(kind, xw, n, yw, m)).all()
    else:
        rows = np.unique(np.concatenate([np.arange(64), np.arange(m - 64, m),
                                         np.random.default_rng(m).integers(0, m, 96)]))
        got = ((z[rows >> 6] >> (rows & 63).astype(np.uint64)) & np.uint64(1)).astype(np.uint8)
        fn = {T: lambda r: oracle.toeplitz_rows(xw, n, yw, m, r),
              C: lambda r: oracle.circulant_rows(xw, n, yw, m, r),
              D: lambda r: oracle.dodis_rows(xw, yw, n, m, r)}[kind]
        assert (got == fn(rows)).all()


def test_cluster_path_equals_goldilocks_path(cm_ctx):
    # the same extractions through the Goldilocks passes (another field, other
    # kernels) give the same bits
    gl = native.Context(0, field=native.FIELD_GOLDILOCKS)
    try:
        for kind, n, m in [(T, 2 ** 16, 2 ** 15), (T, 65537, 65536), (C, na(60000) - 1, 12345),
                           (D, na(70000), 40001)]:
            xw, yw, z, _ = run(cm_ctx, kind, n, m, 9100 + m % 97)
            x, y = to_dev(xw), to_dev(yw)
            ref = {T: lambda: gl.toeplitz(x, n, y, m), C: lambda: gl.circulant(x, n, y, m),
                   D: lambda: gl.dodis(x, y, n, m)}[kind]()
            assert (z == from_dev(ref)).all(), (kind, n, m)
    finally:
        gl.close()


@pytest.mark.parametrize("P,m", [(20000, 7000), (70000, 40001)])
def test_cluster_path_dodis_precondition(cm_ctx, P, m):
    P = na(P)
    x = to_dev(np.zeros(native.words(P), dtype=np.uint64))
    y = to_dev(inputs.bernoulli_half(5, P))
    z = cm_ctx.dodis(x, y, P, m)
    assert cm_ctx.device_status()[0] == native.CM_EPRECOND
    assert (from_dev(z) == 0).all()


# 2^17 products (16-CTA clusters): every window position class (lo = 0, the
# wrap at position 0, m = 1, m = L - K + 1, ragged ends)
WINDOW_CASES = [
    (T, 2 ** 16 + 1, 2 ** 16),            # lo = 2^16, m = 2^16: K + m - 1 = 2^17 exactly
    (T, 65537, 1),                        # m = 1
    (T, 70001, 20000),                    # ragged
    (T, 1, 2 ** 17),                      # n = 1 (lo = 0): z = y
    (C, na(66000) - 1, 33000),
    (D, na(66000), 30001),
]


@pytest.mark.parametrize("kind,n,m", WINDOW_CASES)
def test_2p17_window_cases_match_oracle(cm_ctx, kind, n, m):
    info = native.plan_query(kind, n, m)
    assert info["transform_length"] == 2 ** 17 and info["products"] == 1, info
    xw, yw, z, prof = run(cm_ctx, kind, n, m, 7300 + n % 1000 + m % 71)
    assert prof.get("k_cluster_f25", (0,))[0] == 1, prof
    if m & 63:
        assert int(z[-1]) >> (m & 63) == 0
    if m <= 40000:
        assert (z == want(kind, xw, n, yw, m)).all()
    else:
        rows = np.unique(np.concatenate([np.arange(200), np.arange(m - 200, m),
                                         np.random.default_rng(m).integers(0, m, 200)]))
        got = ((z[rows >> 6] >> (rows & 63).astype(np.uint64)) & np.uint64(1)).astype(np.uint8)
        fn = {T: lambda r: oracle.toeplitz_rows(xw, n, yw, m, r),
              C: lambda r: oracle.circulant_rows(xw, n, yw, m, r),
              D: lambda r: oracle.dodis_rows(xw, yw, n, m, r)}[kind]
        assert (got == fn(rows)).all()
    assert cm_ctx.device_status() == (native.CM_OK, 0)


def test_cluster_path_repeated_calls_and_streams(cm_ctx):
    # back-to-back calls and calls on two streams give the same bits every time
    import torch
    n, m = 2 ** 16, 2 ** 15
    xw, yw = inputs.bernoulli_half(7501, n), inputs.bernoulli_half(7502, n + m - 1)
    x, y = to_dev(xw), to_dev(yw)
    ref = from_dev(cm_ctx.toeplitz(x, n, y, m))
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = []
    for s in (s1, s2, s1, s2):
        with torch.cuda.stream(s):
            outs.append(cm_ctx.toeplitz(x, n, y, m))
    torch.cuda.synchronize()
    for z in outs:
        assert (from_dev(z) == ref).all()
    rows = np.arange(0, m, 97)
    got = ((ref[rows >> 6] >> (rows & 63).astype(np.uint64)) & np.uint64(1)).astype(np.uint8)
    assert (got == oracle.toeplitz_rows(xw, n, yw, m, rows)).all()
