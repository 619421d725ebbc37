"""The field routines of the CUDA path, compiled for the host with g++.

Goldilocks (csrc/gl.cuh) against 128-bit integer arithmetic: add, sub, the
128-bit reduction, multiplication by 2^s (the shift twiddles, 0 <= s <= 96),
and the root structure (g of order 2^32 with g^(2^26) = 8, L^-1).  The 32-bit
field of q = 3 * 2^30 + 1 (csrc/f30.cuh) against plain 64-bit modular
arithmetic: primality, the generator and the root of order 2^30, add, sub, the
Montgomery product, the sub-transform twiddles and the L^-1 constant.  The
lazily reduced field of q = 5 * 2^25 + 1 (csrc/f25.cuh) likewise, with the
value ranges its kernels rely on, and its register DFT modelled step for step."""

import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2402_09481_gb300", "csrc")


def test_field_routines(tmp_path):
    exe = tmp_path / "field_check"
    r = subprocess.run(["g++", "-O2", "-std=c++17", f"-I{CSRC}", os.path.join(HERE, "field_check.cpp"),
                        "-o", str(exe)], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stderr)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "field_check: ok" in r.stdout


def test_field30_routines(tmp_path):
    exe = tmp_path / "field30_check"
    r = subprocess.run(["g++", "-O2", "-std=c++17", f"-I{CSRC}", os.path.join(HERE, "field30_check.cpp"),
                        "-o", str(exe)], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stderr)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "field30_check: ok" in r.stdout


def test_field25_routines(tmp_path):
    exe = tmp_path / "field25_check"
    r = subprocess.run(["g++", "-O2", "-std=c++17", f"-I{CSRC}", os.path.join(HERE, "field25_check.cpp"),
                        "-o", str(exe)], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stderr)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "field25_check: ok" in r.stdout


def f25_b0_bound(lq, s):
    # block 0's input bound (units of q) at stage s, as dft_reg_f25 plans it:
    # double it (no reduction of hi) while a doubled bound plus 2 per remaining
    # stage stays within 24, else reduce hi and add 2
    b = 2
    for j in range(s):
        b = 2 * b if 2 * b + 2 * (lq - 1 - j) <= 24 else b + 2
    return b


def test_lazy_radix_dft_model():
    # The register sub-transform of the lazily reduced field (dft_reg_f25):
    # Cooley-Tukey butterflies on natural-order input, stage s splitting block
    # b with zeta = omega_(2^(s+1))^bitrev_s(b), give X[k] at position
    # bitrev(k); block 0 (zeta = 1) adds hi unreduced while its bound allows.
    # From inputs in [0, 2q) every intermediate stays below the planned bound
    # (4, 8, 16, 18, 20 q for LQ = 1 .. 5) < 25 q < 2^32.  Modelled step for
    # step with exact integers.
    import random
    q = 5 * 2 ** 25 + 1
    w32 = pow(243, 2 ** 20, q)
    mu = 2 ** 32 // q

    def red(x):
        return x - ((x * mu) >> 32) * q

    def shoup(x, w):
        return (x * w - ((x * ((w << 32) // q)) >> 32) * q) % 2 ** 32

    def brv(k, lg):
        return int(format(k, f"0{lg}b")[::-1], 2) if lg else 0

    rng = random.Random(25)
    for lq in range(1, 6):
        rd = 1 << lq
        wr = pow(w32, 32 // rd, q)
        for _ in range(300):
            v = [rng.choice([0, 1, q, 2 * q - 1, rng.randrange(2 * q)]) for _ in range(rd)]
            x = list(v)
            final = f25_b0_bound(lq, lq)
            assert final == [4, 8, 16, 18, 20][lq - 1]
            for s in range(lq):
                ln = rd >> (s + 1)
                bb = f25_b0_bound(lq, s)
                reduce0 = s > 0 and 2 * bb + 2 * (lq - 1 - s) > 24
                for b in range(1 << s):
                    zeta = pow(w32, (32 >> (s + 1)) * brv(b, s), q)
                    for j in range(ln):
                        i0 = b * 2 * ln + j
                        i1 = i0 + ln
                        if b == 0 and not reduce0:
                            t, add = v[i1], bb * q
                            assert max(v[i0], v[i1]) < bb * q
                        else:
                            t, add = (red(v[i1]) if b == 0 else shoup(v[i1], zeta)), 2 * q
                            assert t < 2 * q
                        v[i0], v[i1] = v[i0] + t, v[i0] - t + add
                        assert 0 <= v[i1] and max(v[i0], v[i1]) < final * q < 2 ** 32
            for k in range(rd):
                assert v[brv(k, lq)] % q == sum(x[j] * pow(wr, j * k, q) for j in range(rd)) % q


def test_radix16_bit_table_identity():
    # The first forward step on 0/1 inputs (32-bit field) reads its length-16
    # DFTs from a table: w = omega_16 = g30^(2^26) (the square of the
    # sub-transform root omega_32 = g30^(2^25)), w^8 = -1, so
    # X_k = T_k(b_0..b_7) + (-1)^k T_k(b_8..b_15), T_k(p) = sum_{j in p} w^(jk).
    import random
    q = 3 * 2 ** 30 + 1
    w = pow(125, 2 ** 26, q)
    assert pow(w, 8, q) == q - 1 and pow(w, 16, q) == 1
    T = [[sum(pow(w, j * k % 16, q) for j in range(8) if p >> j & 1) % q for p in range(256)] for k in range(16)]
    rng = random.Random(16)
    for p in [0, 1, 0xFFFF, 0x8000, 0x00FF, 0xFF00] + [rng.getrandbits(16) for _ in range(300)]:
        b = [(p >> i) & 1 for i in range(16)]
        for k in range(16):
            want = sum(b[i] * pow(w, i * k, q) for i in range(16)) % q
            got = (T[k][p & 255] + (q - T[k][p >> 8] if k & 1 else T[k][p >> 8])) % q
            assert got == want, (p, k)


def test_pack_multiply_gathers_four_parity_bytes():
    # k_pack: for 4 bytes b0..b3 in {0, 1} (little-endian word x), byte 3 of
    # x * 0x01020408 (mod 2^32) is b0 + 2 b1 + 4 b2 + 8 b3: no carry reaches it
    for p in range(16):
        b = [(p >> i) & 1 for i in range(4)]
        x = b[0] | b[1] << 8 | b[2] << 16 | b[3] << 24
        assert ((x * 0x01020408) & 0xFFFFFFFF) >> 24 == p
