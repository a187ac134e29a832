"""The compile-time twiddles of the constant-twiddle sphere transforms (csrc/twiddle_const.cuh),
compiled on the host by tests/twiddle_check.cpp: every FP32 constant the kernels take for
cos(2 pi q / n) and sin(2 pi q / n), at every transform size that has them, is the FP32 value
nearest to the exact cosine or sine (computed with 60 significant digits), and the constants
repeat with period n in q."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SIZES = (12, 16, 18, 20, 24, 27)   # the n2 = n3 sizes the constant-twiddle kernel is compiled for


def _nearest_f32(c, x, mp):
    """c (an FP32 value) is at least as close to x as both FP32 neighbours of c."""
    c32 = np.float32(c)
    if float(c32) != c:
        return False
    d = abs(mp.mpf(c) - x)
    for toward in (np.float32(np.inf), np.float32(-np.inf)):
        nb = float(np.nextafter(c32, toward))
        if abs(mp.mpf(nb) - x) < d:
            return False
    return True


def test_constant_twiddles_are_correctly_rounded():
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = 60
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    out_dir = os.path.join(ROOT, "tests", "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "twiddle_check")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_1810_07772_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "twiddle_check.cpp"), "-o", exe], check=True, timeout=300)
    lines = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=60).stdout.split("\n")
    seen = {}
    for ln in filter(None, lines):
        n, q, cs, ss = ln.split()
        n, q = int(n), int(q)
        c, s = float.fromhex(cs), float.fromhex(ss)
        angle = 2 * mp.pi * q / n
        assert _nearest_f32(c, mp.cos(angle), mp), (n, q, "cos", c)
        assert _nearest_f32(s, mp.sin(angle), mp), (n, q, "sin", s)
        if q >= n:
            assert (c, s) == seen[(n, q - n)]          # the integer reduction: period n, bit for bit
        seen[(n, q)] = (c, s)
    assert sorted({n for n, _ in seen}) == list(SIZES)
    assert len(seen) == sum(2 * n for n in SIZES)
    # the exact zeros and units of the quarter turns
    for n in (12, 16, 20, 24):
        assert seen[(n, n // 4)] == (0.0, 1.0) and seen[(n, n // 2)] == (-1.0, 0.0)
