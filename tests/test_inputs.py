"""The seeded input generator: SplitMix64 counter mode."""

import numpy as np

from paper_2402_09481_gb300 import inputs


def test_splitmix64_published_sequence():
    # SplitMix64 seeded with 0 produces 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
    # 0x06C45D188009454F, ... ; the counter form with key 0 is that sequence.
    w = inputs.counter_words(0, 0, 3)
    assert [int(v) for v in w] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_streams_are_seekable_and_masked():
    a = inputs.stream_words(7, 100)
    b = inputs.stream_words(7, 40, first=60)
    assert (a[60:] == b).all()
    w = inputs.bernoulli_half(1, 100)
    assert w.size == 2 and int(w[1]) >> 36 == 0


def test_bias():
    w = inputs.bernoulli(5, 1 << 16)
    ones = int(np.unpackbits(w.view(np.uint8)).sum())
    assert abs(ones / (1 << 16) - 0.8) < 0.01
    h = inputs.bernoulli_half(5, 1 << 16)
    ones = int(np.unpackbits(h.view(np.uint8)).sum())
    assert abs(ones / (1 << 16) - 0.5) < 0.01


def test_loguniform_range():
    n = inputs.loguniform_lengths(1, 4096, 10, 22)
    assert n.min() >= 1024 and n.max() < (1 << 22)
