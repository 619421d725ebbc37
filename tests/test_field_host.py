"""The field routines of the CUDA path, compiled for the host with g++.

Goldilocks (csrc/gl.cuh) against 128-bit integer arithmetic: add, sub, the
128-bit reduction, multiplication by 2^s (the shift twiddles, 0 <= s <= 96),
and the root structure (g of order 2^32 with g^(2^26) = 8, L^-1).  The 32-bit
field of q = 3 * 2^30 + 1 (csrc/f30.cuh) against plain 64-bit modular
arithmetic: primality, the generator and the root of order 2^30, add, sub, the
Montgomery product, the sub-transform twiddles and the L^-1 constant."""

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
