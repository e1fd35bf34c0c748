"""Host-compiled checks of device logic (no GPU): the production headers are
compiled as host code with nvcc.

* The band kernel's triangle items: the compact enumeration (cumulative
  table, binary search, column range) equals the skipping raster, tile for
  tile, over every small geometry (tests/hostcheck/tri_enum.cu).
* The CRT reconstruction's rounding of the exact integer Z 2^s to dd
  (bigfloat.cuh): against exact rationals, hi is the nearest binary64 of the
  value when Z has at most 128 significant bits, and |hi + lo - Z 2^s| stays
  within (2^-106 + 2^-126) |Z 2^s| (plus the subnormal spacing), with
  overflow to a correctly signed infinity.
"""
from __future__ import annotations

import ctypes
import math
import os
import random
import shutil
import subprocess
from fractions import Fraction

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2109_13406_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")


def _nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        pytest.skip("nvcc not available")
    return path


def _build(src, out, shared):
    cmd = [_nvcc(), "-O2", "-std=c++17", "-x", "cu", "-I", CSRC, "-I", INCLUDE, src, "-o", out]
    if shared:
        cmd[1:1] = ["-shared", "-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]


def test_triangle_items_match_the_skipping_raster(tmp_path):
    exe = str(tmp_path / "tri_enum")
    _build(os.path.join(HERE, "hostcheck", "tri_enum.cu"), exe, shared=False)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    cases, bad = (int(x) for x in r.stdout.split()[1::2])
    assert cases > 3000 and bad == 0


def test_words_to_dd_rounding(tmp_path):
    so = str(tmp_path / "words_dd.so")
    _build(os.path.join(HERE, "hostcheck", "words_dd.cu"), so, shared=True)
    lib = ctypes.CDLL(so)
    U8 = ctypes.c_uint32 * 8
    D2 = ctypes.c_double * 2
    lib.words_to_dd.argtypes = [U8, ctypes.c_uint32, ctypes.c_int, D2]
    g = random.Random(11)
    for it in range(20000):
        nbits = g.choice([1, 31, 32, 33, 53, 54, 64, 105, 106, 107, 127, 128, 129, 200, 256])
        Z = g.getrandbits(nbits) | (1 << (nbits - 1))
        if g.random() < 0.1:
            Z = (1 << nbits) - 1                       # all ones: the rounding carries
        s = g.choice([g.randint(-300, 50), g.randint(-1300, -1000), g.randint(800, 1100)])
        neg = g.random() < 0.5
        out = D2()
        lib.words_to_dd(U8(*[(Z >> (32 * t)) & 0xFFFFFFFF for t in range(8)]), int(neg), s, out)
        x = Fraction(Z) * Fraction(2) ** s * (-1 if neg else 1)
        if abs(x) >= Fraction(2) ** 1024 * (1 - Fraction(2) ** -54):
            assert math.isinf(out[0]) and (out[0] < 0) == neg
            continue
        err = abs(Fraction(out[0]) + Fraction(out[1]) - x)
        assert err <= abs(x) * (Fraction(2) ** -106 + Fraction(2) ** -126) + Fraction(2) ** -1074
        if Z.bit_length() <= 128 and abs(x) > Fraction(2) ** -900:
            assert out[0] == float(x)
