"""cm_compose (Section "Composing extractors") against the two oracle calls
chained: the two-source output s = Ext_1(x, y), then the seeded extraction
t = Ext_2(first n2 bits of y, seed = first bits of s); z = s followed by t."""

import numpy as np
import pytest
import torch

import oracle
from oracle import extractors as ex
from paper_2402_09481_gb300 import inputs, native
from conftest import from_dev, to_dev

pytestmark = pytest.mark.gpu
T, C, D = native.TOEPLITZ, native.CIRCULANT, native.DODIS


def ybits(kind, n, m):
    return n + m - 1 if kind == T else (n + 1 if kind == C else n)


def prefix(words, nbits):
    """The first nbits of a packed bit string, packed again (bits past nbits 0)."""
    return ex.pack_bits(ex.unpack_bits(words, nbits))


def oracle_ext(kind, xw, n, yw, m):
    if kind == T:
        return oracle.toeplitz_packed(xw, n, yw, m)
    if kind == C:
        return oracle.circulant_packed(xw, n, yw, m)
    return oracle.dodis_packed(xw, yw, n, m)


def oracle_compose(k1, xw, n1, yw, m1, k2, n2, m2):
    s = oracle_ext(k1, xw, n1, yw, m1)
    t = oracle_ext(k2, prefix(yw, n2), n2, prefix(s, ybits(k2, n2, m2)), m2)
    bits = np.concatenate([ex.unpack_bits(s, m1), ex.unpack_bits(t, m2)])
    return ex.pack_bits(bits)


def na(v):
    return oracle.next_na(v)


# (kind1, n1, m1, kind2, n2, m2): m1 ragged and word-aligned, every kind in
# both stages, the seeded stage's seed exactly m1 bits in some cases
CASES = [
    (D, na(20000), 9001, T, 5000, 3000),
    (D, na(20000), 8192, T, 4000, 4193),                  # aligned m1; seed = m1 bits
    (C, na(30000) - 1, 20000, D, na(9000), 4000),
    (T, 12000, 7000, C, na(3000) - 1, 2500),
    (T, 3000, 2048, T, 1000, 1049),                       # seed = m1 bits
    (C, na(600) - 1, 300, T, 200, 50),
    (D, na(40000), 16000, C, na(15000) - 1, na(15000) - 1),  # stage 2 at m = n
]


@pytest.mark.parametrize("k1,n1,m1,k2,n2,m2", CASES)
def test_compose_matches_chained_oracle(cm_ctx, k1, n1, m1, k2, n2, m2):
    seed = 5000 + n1 % 997 + m2
    xw = inputs.bernoulli_half(seed, n1)
    yw = inputs.bernoulli_half(seed + 1, ybits(k1, n1, m1))
    if k1 == D:
        xw[0] = (xw[0] | np.uint64(1)) & ~np.uint64(2)
    if k2 == D:  # stage 2's input is y's prefix: not constant
        yw[0] = (yw[0] | np.uint64(1)) & ~np.uint64(2)
    z = cm_ctx.compose(k1, to_dev(xw), n1, to_dev(yw), m1, k2, n2, m2)
    assert cm_ctx.device_status()[0] == native.CM_OK
    want = oracle_compose(k1, xw, n1, yw, m1, k2, n2, m2)
    assert (from_dev(z) == want).all()
    # the first m1 bits are the two-source output alone
    alone = {T: lambda: cm_ctx.toeplitz(to_dev(xw), n1, to_dev(yw), m1),
             C: lambda: cm_ctx.circulant(to_dev(xw), n1, to_dev(yw), m1),
             D: lambda: cm_ctx.dodis(to_dev(xw), to_dev(yw), n1, m1)}[k1]()
    assert (ex.unpack_bits(from_dev(z), m1) == ex.unpack_bits(from_dev(alone), m1)).all()


def test_compose_tail_bits_zero_and_prefix_only(cm_ctx):
    # bits of z past m1 + m2 are written 0 whatever z held; y bits past n2 do
    # not reach stage 2 (flipping them changes s only through stage 1)
    k1, n1, m1, k2, n2, m2 = T, 5000, 3001, T, 1500, 1000
    xw = inputs.bernoulli_half(71, n1)
    yw = inputs.bernoulli_half(72, ybits(k1, n1, m1))
    z = torch.full((native.words(m1 + m2),), -1, dtype=torch.int64, device="cuda")
    cm_ctx.compose(k1, to_dev(xw), n1, to_dev(yw), m1, k2, n2, m2, z=z)
    zw = from_dev(z)
    tail = (m1 + m2) % 64
    assert tail == 0 or (zw[-1] >> np.uint64(tail)) == 0
    assert (zw == oracle_compose(k1, xw, n1, yw, m1, k2, n2, m2)).all()


def test_compose_rejects_bad_lengths(cm_ctx):
    xw = to_dev(inputs.bernoulli_half(81, 4000))
    yw = to_dev(inputs.bernoulli_half(82, 4000 + 2000 - 1))
    z = torch.zeros(native.words(6000), dtype=torch.int64, device="cuda")
    L = native.lib()
    h = cm_ctx.handle
    cases = [
        (T, 4000, 2000, T, 1500, 502),       # seed n2 + m2 - 1 = 2001 > m1
        (T, 4000, 2000, T, 6000, 10),        # n2 past y's 5999 bits
        (T, 4000, 2000, C, 1000, 10),        # 1001 not prime
        (T, 4000, 2000, D, 1009, 1010),      # m2 > n2
        (T, 4000, 2000, 7, 100, 10),         # unknown kind
        (T, 4000, 0, T, 100, 10),            # m1 = 0
        (T, 4000, 2000, T, 100, 0),          # m2 = 0
    ]
    for k1, n1, m1, k2, n2, m2 in cases:
        r = L.cm_compose(h, k1, xw.data_ptr(), n1, yw.data_ptr(), m1, k2, n2, m2, z.data_ptr(), None)
        assert r == native.CM_EINVAL, (k1, n1, m1, k2, n2, m2)
    assert (from_dev(z) == 0).all()  # nothing ran


def test_compose_dodis_precondition_in_stage_two(cm_ctx):
    # stage 2 is Dodis et al. on y's prefix: an all-0 prefix is reported
    P = na(2000)
    n1, m1 = 6000, 3000
    xw = inputs.bernoulli_half(91, n1)
    ybits_all = np.concatenate([np.zeros(P, np.uint8), ex.unpack_bits(inputs.bernoulli_half(92, n1 + m1 - 1),
                                                                      n1 + m1 - 1 - P)])
    yw = ex.pack_bits(ybits_all)
    cm_ctx.compose(T, to_dev(xw), n1, to_dev(yw), m1, D, P, 100)
    assert cm_ctx.device_status()[0] == native.CM_EPRECOND
