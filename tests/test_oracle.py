"""Pins for the CPU oracle: it is checked against facts other than itself.

Each test names what it pins and where the fact comes from in the paper.  The
set is chosen so that a plausible slip in the oracle (a transposed matrix, a
sign flip in an index, a dropped pad bit, a window off by one) fails at least
one of them.
"""

import itertools

import numpy as np
import pytest

import oracle
from oracle import extractors as ex
from paper_2402_09481_gb300 import inputs

RNG = np.random.default_rng(20240214)


def rbits(k):
    return RNG.integers(0, 2, size=k, dtype=np.uint8)


# --------------------------------------------------------------------------- #
# independent restatements of the paper's two algorithms (schoolbook cyclic
# convolution over the integers; no matrices)
# --------------------------------------------------------------------------- #
def cyclic_conv(a, b, L):
    w = [0] * L
    for i, ai in enumerate(a):
        if ai:
            for j, bj in enumerate(b):
                if bj:
                    w[(i + j) % L] += 1
    return w


def alg_toeplitz(u, v, n, m):
    """Alg. toeplitz: L = 2^(floor(log2(2n)) + 1); u'[i] = u[i]; v'[i] = v[i]
    for i < m; v'[L - n + 1 + i] = v[m + i] for i = 0 .. n - 2 (the printed loop
    runs to n - 1 and would read v[n + m - 1], one past the seed); output the
    first m entries of the cyclic convolution, mod 2."""
    L = 1 << (int(np.floor(np.log2(2 * n))) + 1)
    assert L >= n + m - 1, "the paper's L is only valid while m <= n + 1"
    up = [0] * L
    vp = [0] * L
    for i in range(m):
        vp[i] = int(v[i])
    for i in range(n):
        up[i] = int(u[i])
    for i in range(n - 1):
        vp[L - n + 1 + i] = int(v[m + i])
    w = cyclic_conv(up, vp, L)
    return np.array([w[i] & 1 for i in range(m)], dtype=np.uint8)


def alg_dodis(u, v, n, m):
    """Alg. dodis: L = 2^(floor(log2(2n - 2)) + 1); u'[i] = u[(n - i) mod n];
    conv(u', v) read as the cyclic convolution modulo n, i.e. the linear
    convolution folded: w_i = lin_i + lin_{i + n}; output first m, mod 2."""
    L = 1 << (int(np.floor(np.log2(2 * n - 2))) + 1)
    assert L >= 2 * n - 1
    up = [int(u[(n - i) % n]) for i in range(n)]
    lin = cyclic_conv(up, [int(b) for b in v], L)
    w = [lin[i] + (lin[i + n] if i + n < L else 0) for i in range(n)]
    return np.array([w[i] & 1 for i in range(m)], dtype=np.uint8)


# --------------------------------------------------------------------------- #
# the displayed matrices
# --------------------------------------------------------------------------- #
def test_toeplitz_matrix_matches_displayed_corners():
    # Eq. toep: first column y_0..y_{m-1}; first row y_0, y_{n+m-2}, ..., y_m.
    n, m = 7, 5
    y = np.arange(n + m - 1)  # distinct labels so every entry is identifiable
    T = ex.toeplitz_matrix(y, n, m)
    assert T.shape == (m, n)
    assert list(T[:, 0]) == list(range(m))
    assert list(T[0, :]) == [0] + list(range(n + m - 2, m - 1, -1))
    # constant along diagonals (Toeplitz structure)
    for i in range(1, m):
        for j in range(1, n):
            assert T[i, j] == T[i - 1, j - 1]


def test_circulant_matrix_matches_displayed_rows():
    # Eq. circ-matrix: row 0 = x', row 1 = x'_{n-1}, x'_0, ..., last row starts x'_1.
    c = np.arange(6)
    C = ex.circulant_matrix(c)
    assert list(C[0]) == [0, 1, 2, 3, 4, 5]
    assert list(C[1]) == [5, 0, 1, 2, 3, 4]
    assert list(C[-1]) == [1, 2, 3, 4, 5, 0]


def test_dodis_matrix_display_and_equals_circ():
    x = np.arange(5)
    D = ex.dodis_matrix(x)
    assert list(D[0]) == [0, 1, 2, 3, 4]
    assert list(D[1]) == [4, 0, 1, 2, 3]
    assert list(D[2]) == [3, 4, 0, 1, 2]
    assert list(D[-1]) == [1, 2, 3, 4, 0]
    assert (D == ex.circulant_matrix(x)).all()


# --------------------------------------------------------------------------- #
# brute force against the paper's algorithms
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("n,m", [(1, 1), (2, 1), (2, 2), (3, 2), (3, 3), (4, 1), (4, 3), (4, 4)])
def test_toeplitz_exhaustive_vs_algorithm(n, m):
    for xb in itertools.product((0, 1), repeat=n):
        for yb in itertools.product((0, 1), repeat=n + m - 1):
            x = np.array(xb, dtype=np.uint8)
            y = np.array(yb, dtype=np.uint8)
            assert (oracle.toeplitz(x, y, n, m) == alg_toeplitz(x, y, n, m)).all()


@pytest.mark.parametrize("P", [3, 5])
def test_dodis_circulant_exhaustive_vs_algorithm(P):
    for xb in itertools.product((0, 1), repeat=P):
        x = np.array(xb, dtype=np.uint8)
        for yb in itertools.product((0, 1), repeat=P):
            y = np.array(yb, dtype=np.uint8)
            for m in range(1, P + 1):
                if x.min() != x.max():
                    assert (oracle.dodis(x, y, P, m) == alg_dodis(x, y, P, m)).all()
                if m <= P - 1 and xb[-1] == 0:
                    # Circulant pads x with one zero: Circulant(x[:-1], y) = Dodis-form with [x, 0]
                    assert (oracle.circulant(x[:-1], y, P - 1, m)
                            == alg_dodis(x, y, P, m)).all()


@pytest.mark.parametrize("n,m", [(8, 8), (13, 5), (20, 31), (24, 24)])
def test_toeplitz_random_vs_algorithm(n, m):
    for _ in range(20):
        x, y = rbits(n), rbits(n + m - 1)
        if m <= n + 1:
            assert (oracle.toeplitz(x, y, n, m) == alg_toeplitz(x, y, n, m)).all()
        # the embedding of Eq. toeplitz-embed: toep(y) is the top-left block of
        # circ(y_0, y_{n+m-2}, ..., y_1), applied to [x, 0^{m-1}]
        N = n + m - 1
        gen = np.array([y[(-k) % N] for k in range(N)], dtype=np.uint8)
        emb = ex.gf2_matvec(ex.circulant_matrix(gen), np.concatenate([x, np.zeros(m - 1, np.uint8)]))
        assert (emb[:m] == oracle.toeplitz(x, y, n, m)).all()


@pytest.mark.parametrize("P", [11, 13, 19, 29, 61])
def test_dodis_random_vs_algorithm(P):
    for _ in range(10):
        x, y = rbits(P), rbits(P)
        if x.min() == x.max():
            continue
        for m in (1, P // 2, P):
            assert (oracle.dodis(x, y, P, m) == alg_dodis(x, y, P, m)).all()


def test_dodis_convolution_form():
    # Dodis(x,y)_i = sum_j R(x)_{(i-j) mod n} y_j with R(x) = x_0, x_{n-1}, ..., x_1
    n = 13
    x, y = rbits(n), rbits(n)
    x[0], x[1] = 0, 1
    R = np.array([x[(-k) % n] for k in range(n)])
    z = [sum(int(R[(i - j) % n]) * int(y[j]) for j in range(n)) & 1 for i in range(n)]
    assert list(oracle.dodis(x, y, n, n)) == z


def test_dodis_shift_matrix_form_is_reversed_order():
    # Eq. DodisOUT with A_1 the displayed cyclic shift (row k = e_{k+1}) and
    # A_i = A_1^i yields the matrix-form outputs in the order z_0, z_{n-1}, ...;
    # the matrix / convolution form is the one the algorithm computes.
    n = 11
    x, y = rbits(n), rbits(n)
    x[0], x[1] = 1, 0
    A1 = np.zeros((n, n), dtype=np.int64)
    for k in range(n):
        A1[k, (k + 1) % n] = 1
    Ai = np.eye(n, dtype=np.int64)
    zA = []
    for _ in range(n):
        zA.append(int((Ai @ x) @ y) & 1)
        Ai = Ai @ A1
    z = oracle.dodis(x, y, n, n)
    assert zA == [int(z[(-i) % n]) for i in range(n)]


# --------------------------------------------------------------------------- #
# closed forms for unit vectors
# --------------------------------------------------------------------------- #
def unit(k, i):
    e = np.zeros(k, dtype=np.uint8)
    e[i] = 1
    return e


def test_unit_vector_closed_forms():
    n, m = 9, 6
    N = n + m - 1
    y = rbits(N)
    for j in range(n):
        z = oracle.toeplitz(unit(n, j), y, n, m)
        assert list(z) == [int(y[(i - j) % N]) for i in range(m)]
    P = 13
    x, yy = rbits(P - 1), rbits(P)
    xp = np.concatenate([x, [0]])
    # Circulant with y = e_j: z_i = x'[(j - i) mod P]
    for j in range(P):
        z = oracle.circulant(x, unit(P, j), P - 1, P - 1)
        assert list(z) == [int(xp[(j - i) % P]) for i in range(P - 1)]
    # Circulant / Dodis with x = e_0: z = y_{0:m-1}
    assert list(oracle.circulant(unit(P - 1, 0), yy, P - 1, 7)) == list(yy[:7])
    assert list(oracle.dodis(unit(P, 0), yy, P, P)) == list(yy)


# --------------------------------------------------------------------------- #
# linearity and shift structure
# --------------------------------------------------------------------------- #
def test_bilinearity():
    n, m = 23, 17
    for _ in range(10):
        x1, x2, y1, y2 = rbits(n), rbits(n), rbits(n + m - 1), rbits(n + m - 1)
        T = oracle.toeplitz
        assert (T(x1 ^ x2, y1, n, m) == T(x1, y1, n, m) ^ T(x2, y1, n, m)).all()
        assert (T(x1, y1 ^ y2, n, m) == T(x1, y1, n, m) ^ T(x1, y2, n, m)).all()
    P = 29
    for _ in range(10):
        a, b, c, d = rbits(P - 1), rbits(P - 1), rbits(P), rbits(P)
        C = oracle.circulant
        assert (C(a ^ b, c, P - 1, 11) == C(a, c, P - 1, 11) ^ C(b, c, P - 1, 11)).all()
        assert (C(a, c ^ d, P - 1, 11) == C(a, c, P - 1, 11) ^ C(a, d, P - 1, 11)).all()


def test_shift_structure():
    P = 19
    x, y = rbits(P), rbits(P)
    x[0], x[1] = 1, 0
    # rotating the seed right by one rotates the (full-length) output right by one
    z = oracle.dodis(x, y, P, P)
    z_rot = oracle.dodis(x, np.roll(y, 1), P, P)
    assert (z_rot == np.roll(z, 1)).all()
    zc = oracle.circulant(x[:-1], y, P - 1, P - 1)
    zc_rot = oracle.circulant(x[:-1], np.roll(y, 1), P - 1, P - 1)
    assert (zc_rot[1:] == zc[:-1]).all()
    # Toeplitz: with x_{n-1} = 0, shifting x down by one shifts the output down by one
    n, m = 15, 9
    xt, yt = rbits(n), rbits(n + m - 1)
    xt[-1] = 0
    zt = oracle.toeplitz(xt, yt, n, m)
    zt2 = oracle.toeplitz(np.concatenate([[0], xt[:-1]]).astype(np.uint8), yt, n, m)
    assert (zt2[1:] == zt[:-1]).all()


# --------------------------------------------------------------------------- #
# Thm. 2-univ and the rank lemmas (exact counts)
# --------------------------------------------------------------------------- #
def gf2_rank(M):
    M = (np.array(M, dtype=np.uint8) & 1).copy()
    r = 0
    rows, cols = M.shape
    for c in range(cols):
        piv = next((i for i in range(r, rows) if M[i, c]), None)
        if piv is None:
            continue
        M[[r, piv]] = M[[piv, r]]
        for i in range(rows):
            if i != r and M[i, c]:
                M[i] ^= M[r]
        r += 1
        if r == rows:
            break
    return r


@pytest.mark.parametrize("P,m", [(11, 6), (11, 10), (13, 4), (5, 4)])
def test_two_universality_exact_count(P, m):
    # Thm. 2-univ: for x != x~, exactly 2^(P-m) seeds y make the outputs collide.
    Y = np.array(list(itertools.product((0, 1), repeat=P)), dtype=np.uint8)
    for _ in range(6):
        x, xt = rbits(P - 1), rbits(P - 1)
        if (x == xt).all():
            xt[0] ^= 1
        xp = np.concatenate([x, [0]])
        xtp = np.concatenate([xt, [0]])
        Cx = ex.circulant_matrix(xp)[:m].astype(np.int64)
        Ct = ex.circulant_matrix(xtp)[:m].astype(np.int64)
        Zx = (Y.astype(np.int64) @ Cx.T) & 1
        Zt = (Y.astype(np.int64) @ Ct.T) & 1
        collide = int((Zx == Zt).all(axis=1).sum())
        assert collide == 2 ** (P - m)
        # and the oracle's own entry point agrees on a few seeds
        for y in Y[:: max(1, len(Y) // 16)]:
            assert (oracle.circulant(x, y, P - 1, m) == Zx[int(''.join(map(str, y)), 2)]).all()


@pytest.mark.parametrize("P", [3, 5, 11, 13])
def test_rank_lemmas(P):
    # Lemma circ-row-rank: rank(circ(d')) >= P - 1 for d' not all-0 / all-1;
    # Lemma fullrank: any m <= P - 1 rows have full row rank.
    for db in itertools.product((0, 1), repeat=P):
        d = np.array(db, dtype=np.uint8)
        if d.min() == d.max():
            continue
        C = ex.circulant_matrix(d)
        assert gf2_rank(C) >= P - 1
        rows = RNG.choice(P, size=P - 1, replace=False)
        assert gf2_rank(C[rows]) == P - 1
    # P = 7 has order(2) = 3: the lemma's hypothesis matters
    d = np.array([1, 1, 0, 1, 0, 0, 0], dtype=np.uint8)
    assert gf2_rank(ex.circulant_matrix(d)) < 6


# --------------------------------------------------------------------------- #
# tier 2 (packed rows) against tier 1 (explicit matrices)
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("n,m", [(1, 1), (5, 3), (63, 2), (64, 64), (65, 100), (200, 129), (300, 1)])
def test_toeplitz_rows_match_matrix(n, m):
    x, y = rbits(n), rbits(n + m - 1)
    z = oracle.toeplitz(x, y, n, m)
    zp = oracle.toeplitz_packed(ex.pack_bits(x), n, ex.pack_bits(y), m)
    assert (ex.unpack_bits(zp, m) == z).all()
    rows = RNG.choice(m, size=min(m, 7), replace=False)
    assert (oracle.toeplitz_rows(ex.pack_bits(x), n, ex.pack_bits(y), m, rows) == z[rows]).all()


@pytest.mark.parametrize("P", [3, 11, 61, 67, 131, 197])
def test_circulant_dodis_rows_match_matrix(P):
    x, y = rbits(P), rbits(P)
    x[0], x[1] = 0, 1
    for m in (1, P // 3 + 1, P - 1):
        zc = oracle.circulant(x[:-1], y, P - 1, m)
        zcp = oracle.circulant_packed(ex.pack_bits(x[:-1]), P - 1, ex.pack_bits(y), m)
        assert (ex.unpack_bits(zcp, m) == zc).all()
    for m in (1, P):
        zd = oracle.dodis(x, y, P, m)
        zdp = oracle.dodis_packed(ex.pack_bits(x), ex.pack_bits(y), P, m)
        assert (ex.unpack_bits(zdp, m) == zd).all()


def test_tail_bits_ignored_and_zeroed():
    n, m = 70, 10
    x, y = rbits(n), rbits(n + m - 1)
    xw, yw = ex.pack_bits(x), ex.pack_bits(y)
    xw_dirty, yw_dirty = xw.copy(), yw.copy()
    xw_dirty[-1] |= np.uint64(0xFFFF) << np.uint64(48)
    yw_dirty[-1] |= np.uint64(1) << np.uint64(63)
    z1 = oracle.toeplitz_packed(xw, n, yw, m)
    z2 = oracle.toeplitz_packed(xw_dirty, n, yw_dirty, m)
    assert (z1 == z2).all()
    assert int(z1[-1]) >> m == 0


def test_preconditions():
    with pytest.raises(oracle.DodisPreconditionError):
        oracle.dodis(np.zeros(5, np.uint8), rbits(5), 5, 2)
    with pytest.raises(oracle.DodisPreconditionError):
        oracle.dodis(np.ones(5, np.uint8), rbits(5), 5, 2)
    # Circulant allows x = 0 (the pad bit makes x' differ from all-one anyway)
    assert not oracle.circulant(np.zeros(4, np.uint8), rbits(5), 4, 4).any()
    with pytest.raises(ValueError):
        oracle.circulant(rbits(4), rbits(5), 4, 5)


def test_pack_roundtrip_and_generator_bits():
    for k in (1, 63, 64, 65, 1000):
        b = rbits(k)
        assert (ex.unpack_bits(ex.pack_bits(b), k) == b).all()
    w = inputs.bernoulli_half(3, 130)
    assert int(w[-1]) >> 2 == 0


def test_rows_at_workload_size_vs_index_formula():
    # tier 2 at the Circulant workload size (P = 16777259) against rows built
    # directly from the index formula of Eq. circ-matrix for a few rows
    P = 16777259
    xw = inputs.bernoulli_half(11, P - 1)
    yw = inputs.bernoulli_half(12, P)
    xp = np.concatenate([ex.unpack_bits(xw, P - 1), np.zeros(1, np.uint8)])
    y = ex.unpack_bits(yw, P).astype(np.int64)
    m = P // 2
    rows = np.array([0, 1, 12345, m - 1])
    got = oracle.circulant_rows(xw, P - 1, yw, m, rows)
    j = np.arange(P)
    for r, g in zip(rows, got):
        assert int(xp[(j - r) % P].astype(np.int64) @ y) & 1 == g
