"""The bit-packed CPU NTT extractor (cpu_ntt.cpp): the CPU baseline that the
benchmark times beside the GPU path.  It shares no code with the GPU library
(paper_2402_09481_gb300) or the oracle; the tests check it against the oracle.

build()   compile cpu_ntt.cpp into cpu_ntt/_build/libcpu_ntt.so (g++, no GPU).
extract() one extraction on host buffers with a given number of threads.
"""

from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpu_ntt.cpp")
LIB = os.path.join(HERE, "_build", "libcpu_ntt.so")
_lib = None

TOEPLITZ, CIRCULANT, DODIS = 0, 1, 2


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cxx = shutil.which("g++") or "g++"
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + ".tmp"
    r = subprocess.run([cxx, "-O3", "-std=c++20", "-pthread", "-shared", "-fPIC", "-o", tmp, SRC],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"g++ failed on cpu_ntt.cpp:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        L.cpu_ntt_extract.restype = ctypes.c_int
        L.cpu_ntt_extract.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                      ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int]
        L.cpu_ntt_prepare.restype = None
        L.cpu_ntt_prepare.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def transform_lg(kind: int, n: int, m: int) -> int:
    K = n + 1 if kind == CIRCULANT else n
    return max(1, (K + m - 2).bit_length())


def prepare(kind: int, n: int, m: int) -> None:
    """Build the root tables of the extraction's transform length (untimed)."""
    lib().cpu_ntt_prepare(transform_lg(kind, n, m))


def extract(kind: int, x_words, n: int, y_words, m: int, threads: int = 1) -> np.ndarray:
    """z (ceil(m / 64) uint64 words) of the extraction on host buffers."""
    x = np.ascontiguousarray(x_words, dtype=np.uint64)
    y = np.ascontiguousarray(y_words, dtype=np.uint64)
    z = np.zeros((m + 63) // 64, dtype=np.uint64)
    rc = lib().cpu_ntt_extract(kind, x.ctypes.data, n, y.ctypes.data, m, z.ctypes.data, int(threads))
    if rc != 0:
        raise ValueError(f"cpu_ntt_extract: invalid arguments (kind {kind}, n {n}, m {m})")
    return z
