"""cm_calibrate: the planner's figures timed on this GPU, kept in the context
and cached per device; extractions under the calibrated planner (including a
calibrated pass split) stay bit-exact."""

import os
import time

import numpy as np
import pytest

import oracle
from paper_2402_09481_gb300 import inputs, native
from conftest import from_dev, to_dev

pytestmark = pytest.mark.gpu
T, C, D = native.TOEPLITZ, native.CIRCULANT, native.DODIS
Q25, Q30, GL = native.FIELD_Q25, native.FIELD_Q30, native.FIELD_GOLDILOCKS


def ybits(kind, n, m):
    return n + m - 1 if kind == T else (n + 1 if kind == C else n)


def extract(ctx, kind, n, m, xw, yw):
    x, y = to_dev(xw), to_dev(yw)
    if kind == T:
        return from_dev(ctx.toeplitz(x, n, y, m))
    if kind == C:
        return from_dev(ctx.circulant(x, n, y, m))
    return from_dev(ctx.dodis(x, y, n, m))


def test_calibrate_measures_and_caches(tmp_path):
    cache = str(tmp_path / "tune.txt")
    ctx = native.Context(0)
    try:
        t0 = time.time()
        ctx.calibrate(cache, max_lg=20)
        t_measure = time.time() - t0
        assert os.path.exists(cache)
        for lg in range(9, 21):
            assert ctx.tune_query(Q25, lg)[0] > 0
        for lg in range(14, 21):
            assert ctx.tune_query(Q30, lg)[0] > 0 and ctx.tune_query(GL, lg)[0] > 0
        for lg in range(14, 18):
            assert ctx.tune_query(Q25, lg)[1] > 0  # the cluster form
        assert ctx.tune_query(Q25, 21)[0] == 0     # past max_lg: the built-in figures
        figs = {(f, lg): ctx.tune_query(f, lg) for f in (Q25, Q30, GL) for lg in range(9, 21)}
    finally:
        ctx.close()
    lines = open(cache).read().splitlines()
    assert lines[0] == "cm-tune 2" and lines[1].startswith("device ")
    # a second context loads the same figures from the cache instead of timing
    ctx2 = native.Context(0)
    try:
        t0 = time.time()
        ctx2.calibrate(cache)
        assert time.time() - t0 < t_measure
        assert {(f, lg): ctx2.tune_query(f, lg) for f in (Q25, Q30, GL) for lg in range(9, 21)} == figs
    finally:
        ctx2.close()


def test_foreign_cache_is_measured_again(tmp_path):
    cache = tmp_path / "tune.txt"
    cache.write_text("cm-tune 2\ndevice Some_Other_GPU 99\ncost 2 12 123.0\n")
    ctx = native.Context(0)
    try:
        ctx.calibrate(str(cache), max_lg=14)
        ms = ctx.tune_query(Q25, 12)[0]
        assert 0 < ms < 123.0
        assert "Some_Other_GPU" not in cache.read_text()
        ctx.calibrate(str(cache), force=True, max_lg=13)  # forced: measured again, file rewritten
        assert ctx.tune_query(Q25, 14)[0] == 0
    finally:
        ctx.close()


CASES = [(T, 1000, 500), (T, 20000, 12000), (T, 2 ** 16, 2 ** 15), (T, 300000, 150001),
         (C, "P40000", 0.5), (D, "P70000", 0.4), (T, 1_500_000, 700_000)]


def resolve(kind, n, m):
    if isinstance(n, str):
        P = oracle.next_na(int(n[1:]))
        n = P - 1 if kind == C else P
        m = max(1, int(m * n))
    return n, m


def test_calibrated_plans_bit_exact():
    ctx = native.Context(0)
    try:
        ctx.calibrate(None, max_lg=22)
        for kind, n, m in CASES:
            n, m = resolve(kind, n, m)
            xw = inputs.bernoulli_half(400 + n % 97, n)
            if kind == D:
                xw[0] = (xw[0] | np.uint64(1)) & ~np.uint64(2)
            yw = inputs.bernoulli_half(401 + n % 89, ybits(kind, n, m))
            z = extract(ctx, kind, n, m, xw, yw)
            if m <= 40000:
                want = {T: oracle.toeplitz_packed, C: oracle.circulant_packed}.get(kind)
                ref = want(xw, n, yw, m) if want else oracle.dodis_packed(xw, yw, n, m)
                assert (z == ref).all(), (kind, n, m)
            else:
                rows = np.unique(np.random.default_rng(m).integers(0, m, 64))
                got = ((z[rows >> 6] >> (rows & 63).astype(np.uint64)) & np.uint64(1)).astype(np.uint8)
                fn = {T: oracle.toeplitz_rows, C: oracle.circulant_rows}.get(kind)
                ref = fn(xw, n, yw, m, rows) if fn else oracle.dodis_rows(xw, yw, n, m, rows)
                assert (got == ref).all(), (kind, n, m)
    finally:
        ctx.close()


@pytest.mark.slow
def test_calibrated_pass_split_bit_exact():
    # two-pass transforms over 3 * 2^30 + 1 with the calibrated first-pass
    # length: the same bits as the Goldilocks single transform
    q30 = native.Context(0, field=Q30, plan_mode=native.PLAN_SINGLE)
    gl = native.Context(0, field=GL, plan_mode=native.PLAN_SINGLE)
    try:
        q30.calibrate(None, max_lg=27)
        for lg in (26, 27):
            ms, _, split = q30.tune_query(Q30, lg)
            assert ms > 0
            rest, d = lg - 13, (lg - 13 + 1) // 2
            assert split in (0, d - 1, d + 1)
        n, m = 2 ** 25 + 12345, 2 ** 25 - 12445   # K + m - 1 = 2^26 - 101
        xw = inputs.bernoulli_half(450, n)
        yw = inputs.bernoulli_half(451, n + m - 1)
        assert (extract(q30, T, n, m, xw, yw) == extract(gl, T, n, m, xw, yw)).all()
    finally:
        q30.close()
        gl.close()
