"""Pins of the Von Neumann oracle (Section "Von Neumann", Alg. vn).

Hand-worked pairs, the loop and array forms against each other on every input
up to 12 bits, the no-output error, the odd trailing bit, and the property the
section states for exchangeable input: given the output length, every output
string is equally likely (checked by exact enumeration for IID bits of several
biases).  Packed forms round-trip through the bit packing.
"""

from itertools import product
import math

import numpy as np
import pytest

from oracle import von_neumann as vn
from oracle.extractors import pack_bits


def test_hand_worked():
    # pairs (0,1) -> 0, (1,0) -> 1, (1,1) -> nothing, (0,0) -> nothing
    assert vn.von_neumann_loop([0, 1, 1, 0]) == [0, 1]
    assert vn.von_neumann_loop([1, 1, 0, 1, 0, 0, 1, 0]) == [0, 1]
    assert vn.von_neumann_loop([1, 0]) == [1]
    # a trailing odd bit belongs to no pair
    assert vn.von_neumann_loop([0, 1, 1]) == [0]
    assert vn.von_neumann_loop([1, 0, 0]) == [1]


@pytest.mark.parametrize("bits", [[], [1], [0, 0], [1, 1, 0, 0], [1] * 9, [0] * 64])
def test_no_output_is_an_error(bits):
    with pytest.raises(vn.VonNeumannNoOutput):
        vn.von_neumann_loop(bits)
    with pytest.raises(vn.VonNeumannNoOutput):
        vn.von_neumann(np.array(bits, dtype=np.uint8))


def test_array_form_equals_loop_exhaustively():
    for n in range(0, 13):
        for bits in product((0, 1), repeat=n):
            try:
                want = vn.von_neumann_loop(bits)
            except vn.VonNeumannNoOutput:
                with pytest.raises(vn.VonNeumannNoOutput):
                    vn.von_neumann(np.array(bits, dtype=np.uint8))
                continue
            got = vn.von_neumann(np.array(bits, dtype=np.uint8))
            assert got.tolist() == want


@pytest.mark.parametrize("p", [0.5, 0.3, 0.85])
def test_output_unbiased_given_length(p):
    # IID input bits with Pr[1] = p: conditioned on the output length L, every
    # L-bit output string has probability C(L) / 2^L (exact enumeration, n = 10)
    n = 10
    prob = {}
    for bits in product((0, 1), repeat=n):
        pr = math.prod(p if b else 1 - p for b in bits)
        try:
            out = tuple(vn.von_neumann_loop(bits))
        except vn.VonNeumannNoOutput:
            continue
        prob[out] = prob.get(out, 0.0) + pr
    by_len = {}
    for out, pr in prob.items():
        by_len.setdefault(len(out), []).append(pr)
    for L, prs in by_len.items():
        assert len(prs) == 2 ** L
        assert max(prs) == pytest.approx(min(prs), rel=1e-12)


def test_packed_matches_unpacked():
    rng = np.random.default_rng(3)
    for n in (2, 63, 64, 65, 127, 128, 1000, 4097):
        b = (rng.random(n) < 0.7).astype(np.uint8)
        b[0], b[1] = 1, 0   # at least one output bit
        words, m = vn.von_neumann_packed(pack_bits(b), n)
        want = vn.von_neumann(b)
        assert m == want.size
        assert (words == pack_bits(want)).all()
        assert vn.von_neumann_count(pack_bits(b), n) == m


def test_word_counts_and_sampled_bits_match_full_output():
    rng = np.random.default_rng(9)
    for n, p in ((1, 0.5), (2, 0.5), (65, 0.5), (1000, 0.1), (4097, 0.93), (20001, 0.5)):
        b = (rng.random(n) < p).astype(np.uint8)
        words = pack_bits(b)
        k = n // 2
        per_pair = (b[0:2 * k:2] != b[1:2 * k:2]).astype(np.int64)
        per_word = np.add.reduceat(per_pair, np.arange(0, k, 32)) if k else np.zeros(0, np.int64)
        assert vn.pair_counts_per_word(words, n).tolist() == per_word.tolist()
        m = int(per_pair.sum())
        if m == 0:
            continue
        full = vn.von_neumann(b)
        pos = rng.integers(0, m, 50)
        got, mm = vn.output_bits_at(words, n, pos)
        assert mm == m and got.tolist() == full[pos].tolist()
