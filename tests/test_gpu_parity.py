"""GPU path vs the CPU oracle, bit for bit, through the C ABI.

Sizes span the single-CTA path (L <= 2^13), the one-pass path (2^14 .. 2^25)
and the two-pass path (L >= 2^26), ragged lengths (not multiples of 64, not
powers of two), the configurations the benchmark times, and the degenerate
cases (m = 1, n = 1, maximal m, L exactly K + m - 1).  Where the oracle can
build every output row the whole output is compared; at the full benchmark
sizes a sample of rows (first, last and random) is compared.
"""

import numpy as np
import pytest
import torch

import oracle
from oracle import extractors as ex
from paper_2402_09481_gb300 import inputs, native
from conftest import from_dev, to_dev

pytestmark = pytest.mark.gpu


def sample_rows(m, k=96, seed=0):
    rng = np.random.default_rng(seed + m)
    head = np.arange(min(m, 32))
    tail = np.arange(max(0, m - 32), m)
    mid = rng.integers(0, m, size=k)
    return np.unique(np.concatenate([head, tail, mid]))


def out_bits(zw, m, rows):
    z = np.asarray(zw, dtype=np.uint64)
    return ((z[rows >> 6] >> (rows & 63).astype(np.uint64)) & np.uint64(1)).astype(np.uint8)


def check_tail(zw, m):
    z = np.asarray(zw, dtype=np.uint64)
    assert z.size == native.words(m)
    if m & 63:
        assert int(z[-1]) >> (m & 63) == 0


# --------------------------------------------------------------------------- #
TOEPLITZ_FULL = [(1, 1), (1, 5), (2, 1), (3, 7), (5, 3), (63, 1), (64, 64), (65, 63),
                 (100, 28), (1000, 1000), (4096, 4097), (8000, 193),
                 (5000, 4000), (20000, 12000), (2 ** 16, 2 ** 15), (100000, 31073)]


@pytest.mark.parametrize("n,m", TOEPLITZ_FULL)
def test_toeplitz_full(cm_ctx, n, m):
    xw = inputs.bernoulli_half(101, n)
    yw = inputs.bernoulli_half(102, n + m - 1)
    z = from_dev(cm_ctx.toeplitz(to_dev(xw), n, to_dev(yw), m))
    check_tail(z, m)
    assert (z == oracle.toeplitz_packed(xw, n, yw, m)).all()


TOEPLITZ_SAMPLED = [(3 * 2 ** 17, 2 ** 17), (2 ** 24, 2 ** 24), (2 ** 25, 2 ** 25 + 1),
                    (12345678, 3456789)]


@pytest.mark.parametrize("n,m", TOEPLITZ_SAMPLED)
def test_toeplitz_sampled(cm_ctx, n, m):
    xw = inputs.bernoulli_half(103, n)
    yw = inputs.bernoulli_half(104, n + m - 1)
    z = from_dev(cm_ctx.toeplitz(to_dev(xw), n, to_dev(yw), m))
    check_tail(z, m)
    rows = sample_rows(m)
    assert (out_bits(z, m, rows) == oracle.toeplitz_rows(xw, n, yw, m, rows)).all()


CIRC_FULL = [3, 5, 11, 13, 61, 67, 197, 1019, 4099, 16411, 131101]


@pytest.mark.parametrize("P", CIRC_FULL)
def test_circulant_full(cm_ctx, P):
    P = oracle.next_na(P)
    n = P - 1
    xw = inputs.bernoulli_half(201, n)
    yw = inputs.bernoulli_half(202, P)
    for m in sorted({1, max(1, n // 2), n}):
        z = from_dev(cm_ctx.circulant(to_dev(xw), n, to_dev(yw), m))
        check_tail(z, m)
        assert (z == oracle.circulant_packed(xw, n, yw, m)).all(), (P, m)


def test_circulant_workload_size(cm_ctx):
    P = 16777259                      # smallest N_A member >= 2^24
    n, m = P - 1, (P - 1) // 2        # m = n/2 as in the benchmark
    xw = inputs.bernoulli_half(1, n)
    yw = inputs.bernoulli_half(2, P)
    z = from_dev(cm_ctx.circulant(to_dev(xw), n, to_dev(yw), m))
    check_tail(z, m)
    rows = sample_rows(m, k=400)
    assert (out_bits(z, m, rows) == oracle.circulant_rows(xw, n, yw, m, rows)).all()


DODIS_FULL = [3, 5, 13, 101, 1019, 4091, 16411, 70001]


@pytest.mark.parametrize("P", DODIS_FULL)
def test_dodis_full(cm_ctx, P):
    n = oracle.next_na(P)
    xw = inputs.bernoulli_half(301, n)
    xw[0] = (xw[0] | np.uint64(1)) & ~np.uint64(2)   # precondition: x not constant
    yw = inputs.bernoulli_half(302, n)
    for m in sorted({1, max(1, (2 * n) // 5), n}):
        z = from_dev(cm_ctx.dodis(to_dev(xw), to_dev(yw), n, m))
        check_tail(z, m)
        assert (z == oracle.dodis_packed(xw, yw, n, m)).all(), (n, m)
    s, f = cm_ctx.device_status()
    assert s == native.CM_OK and f == 0


def test_dodis_biased_source(cm_ctx):
    n = oracle.next_na(50000)
    m = (2 * n) // 5
    xw = inputs.bernoulli(303, n)          # P(1) = 0.8
    yw = inputs.bernoulli_half(304, n)
    z = from_dev(cm_ctx.dodis(to_dev(xw), to_dev(yw), n, m))
    assert (z == oracle.dodis_packed(xw, yw, n, m)).all()


@pytest.mark.parametrize("n", [13, 70001, 1048583])
def test_dodis_precondition(cm_ctx, n):
    n = oracle.next_na(n)
    m = n // 2
    yw = to_dev(inputs.bernoulli_half(305, n))
    for fill in (0, 1):
        bits = np.full(n, fill, dtype=np.uint8)
        xw = to_dev(ex.pack_bits(bits))
        z = cm_ctx.dodis(xw, yw, n, m)
        s, f = cm_ctx.device_status()
        assert s == native.CM_EPRECOND and f & native.FLAG_PRECOND
        assert not from_dev(z).any()
    # the flag was cleared; a valid call reports OK
    xw = to_dev(inputs.bernoulli_half(306, n))
    cm_ctx.dodis(xw, yw, n, m)
    assert cm_ctx.device_status() == (native.CM_OK, 0)


def test_dirty_input_tails_ignored(cm_ctx):
    for (n, m) in ((100, 37), (70000, 30001)):
        xw = inputs.bernoulli_half(401, n)
        yw = inputs.bernoulli_half(402, n + m - 1)
        xd, yd = xw.copy(), yw.copy()
        xd[-1] |= np.uint64(0xFFFF) << np.uint64(48)
        yd[-1] |= np.uint64(1) << np.uint64(63)
        z1 = from_dev(cm_ctx.toeplitz(to_dev(xw), n, to_dev(yw), m))
        z2 = from_dev(cm_ctx.toeplitz(to_dev(xd), n, to_dev(yd), m))
        assert (z1 == z2).all()


def test_invalid_arguments(cm_ctx):
    L = native.lib()
    d = to_dev(np.zeros(4, dtype=np.uint64))
    p = d.data_ptr()
    s = torch.cuda.current_stream().cuda_stream
    h = cm_ctx.handle
    assert L.cm_toeplitz(h, p, 5, p, 0, p, s) == native.CM_EINVAL          # m = 0
    assert L.cm_toeplitz(h, p, 2 ** 40 + 1, p, 5, p, s) == native.CM_EINVAL  # n > 2^40
    assert L.cm_toeplitz(h, p, 5, p, 2 ** 40 + 1, p, s) == native.CM_EINVAL  # m > 2^40
    assert L.cm_circulant(h, p, 6, p, 3, p, s) == native.CM_EINVAL          # 7 not in N_A
    assert L.cm_circulant(h, p, 10, p, 11, p, s) == native.CM_EINVAL        # m > n
    assert L.cm_dodis(h, p, p, 9, 3, p, s) == native.CM_EINVAL              # 9 not prime
    assert L.cm_dodis(h, p, p, 11, 12, p, s) == native.CM_EINVAL
    assert L.cm_toeplitz(h, None, 5, p, 3, p, s) == native.CM_EINVAL        # null pointer
    with pytest.raises(native.CMError):
        cm_ctx.circulant(d, 6, d, 3)


def test_deterministic_and_stream_ordered(cm_ctx):
    n, m = 300000, 150001
    xw = to_dev(inputs.bernoulli_half(501, n))
    yw = to_dev(inputs.bernoulli_half(502, n + m - 1))
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        z1 = cm_ctx.toeplitz(xw, n, yw, m, stream=st)
        z2 = cm_ctx.toeplitz(xw, n, yw, m, stream=st)
    st.synchronize()
    assert torch.equal(z1, z2)
    z3 = cm_ctx.toeplitz(xw, n, yw, m)
    assert torch.equal(z1, z3)


@pytest.mark.slow
def test_dodis_workload_size(cm_ctx):
    n = 1073741789                    # largest N_A member <= 2^30 (L = 2^31)
    m = (2 * n) // 5
    xw = inputs.bernoulli_half(3, n)
    yw = inputs.bernoulli_half(4, n)
    z = from_dev(cm_ctx.dodis(to_dev(xw), to_dev(yw), n, m))
    torch.cuda.empty_cache()
    check_tail(z, m)
    rows = sample_rows(m, k=16)
    assert (out_bits(z, m, rows) == oracle.dodis_rows(xw, yw, n, m, rows)).all()


def test_modmul_rate(cm_ctx):
    # the integer-pipe denominators of the path roofline: positive, and the
    # 32-bit Montgomery product (3 multiply-adds) faster than the Goldilocks
    # product (a 64 x 64-bit multiply in 32-bit pieces and its reduction)
    q30 = native.modmul_rate(0, native.FIELD_Q30)
    q25 = native.modmul_rate(0, native.FIELD_Q25)
    gl = native.modmul_rate(0, native.FIELD_GOLDILOCKS)
    assert 1e11 < gl < q30 < 1e14 and 1e11 < q25 < 1e14
    with pytest.raises(native.CMError):
        native.modmul_rate(0, 7)


def test_field_selftest_device_arithmetic(cm_ctx):
    # the PTX carry-chain arithmetic against the C forms (which the CPU test
    # pins to 128-bit integers), on edge values and 4M random pairs
    assert native.field_selftest(0, 1 << 22, 12345) == 0


# --------------------------------------------------------------------------- #
# The single calls take the lazily reduced field of 5 * 2^25 + 1 for transforms
# up to 2^25, the field of 3 * 2^30 + 1 up to 2^30 and Goldilocks above; a
# context with CM_FIELD_Q30 skips the first, one with CM_FIELD_GOLDILOCKS keeps
# the 64-bit field at every length.  All must give the oracle's bits.
@pytest.fixture(scope="module")
def gl_ctx():
    from paper_2402_09481_gb300 import build
    build.build()
    c = native.Context(0, field=native.FIELD_GOLDILOCKS)
    yield c
    c.close()


@pytest.fixture(scope="module")
def q30_ctx():
    from paper_2402_09481_gb300 import build
    build.build()
    c = native.Context(0, field=native.FIELD_Q30)
    yield c
    c.close()


@pytest.mark.parametrize("kind,n,m", [
    (native.TOEPLITZ, 5, 3), (native.TOEPLITZ, 5000, 4000), (native.TOEPLITZ, 100000, 31073),
    (native.TOEPLITZ, 2 ** 20, 2 ** 19 + 3), (native.TOEPLITZ, 8193, 8192), (native.TOEPLITZ, 2 ** 24, 2 ** 24),
    (native.TOEPLITZ, 9_000_001, 777_777),
    (native.CIRCULANT, "P131101", 0.5), (native.DODIS, "P40000", 0.4), (native.DODIS, "P3000", 0.9),
    (native.CIRCULANT, "P16777259", 0.5),
])
def test_all_fields_match_oracle(gl_ctx, q30_ctx, cm_ctx, kind, n, m):
    if isinstance(n, str):
        P = oracle.next_na(int(n[1:]))
        n = P - 1 if kind == native.CIRCULANT else P
        m = max(1, int(m * n))
    xw = inputs.bernoulli_half(700 + n % 89, n)
    if kind == native.DODIS:
        xw[0] = (xw[0] | np.uint64(1)) & ~np.uint64(2)
    yb = n + m - 1 if kind == native.TOEPLITZ else (n + 1 if kind == native.CIRCULANT else n)
    yw = inputs.bernoulli_half(701 + n % 83, yb)
    outs = []
    for ctx in (gl_ctx, q30_ctx, cm_ctx):
        x, y = to_dev(xw), to_dev(yw)
        if kind == native.TOEPLITZ:
            z = ctx.toeplitz(x, n, y, m)
        elif kind == native.CIRCULANT:
            z = ctx.circulant(x, n, y, m)
        else:
            z = ctx.dodis(x, y, n, m)
        outs.append(from_dev(z))
    if m <= 131100:
        want = {native.TOEPLITZ: lambda: oracle.toeplitz_packed(xw, n, yw, m),
                native.CIRCULANT: lambda: oracle.circulant_packed(xw, n, yw, m),
                native.DODIS: lambda: oracle.dodis_packed(xw, yw, n, m)}[kind]()
        assert (outs[0] == want).all()
    else:
        rows = sample_rows(m)
        got = out_bits(outs[0], m, rows)
        if kind == native.TOEPLITZ:
            assert (got == oracle.toeplitz_rows(xw, n, yw, m, rows)).all()
        elif kind == native.CIRCULANT:
            assert (got == oracle.circulant_rows(xw, n, yw, m, rows)).all()
        else:
            assert (got == oracle.dodis_rows(xw, yw, n, m, rows)).all()
    assert (outs[0] == outs[1]).all() and (outs[0] == outs[2]).all()
