"""Double-float arithmetic of the emulated-FP64 factorizations, checked on the host.

csrc/tjm_df64.cuh is compiled as plain C++ (its functions are host-and-device)
and every operation is compared with exact rational arithmetic on random
operands over a wide exponent range: add, subtract, multiply, divide and sqrt
must be accurate to a few units of 2^-48 relative to the result; the fused
multiply-add uses the sloppy adder, whose error is bounded relative to the
magnitudes of its two summands.
"""
import os
import shutil
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2501_17913_gb300", "csrc")


def _compiler():
    for c in ("g++", "c++", "clang++"):
        if shutil.which(c):
            return c
    pytest.skip("no C++ compiler")


def _words(rng, n, emin=-30, emax=30):
    """n random double-float values (hi, lo) with |lo| <= ulp(hi)/2, as float32 pairs."""
    x = rng.standard_normal(n) * np.exp2(rng.integers(emin, emax, n).astype(float))
    hi = x.astype(np.float32)
    lo = ((x - hi.astype(np.float64)) + rng.standard_normal(n) * np.abs(x) * 2.0 ** -40).astype(np.float32)
    # renormalise so that hi = fl(hi + lo)
    s = (hi.astype(np.float64) + lo.astype(np.float64))
    hi2 = s.astype(np.float32)
    lo2 = (s - hi2.astype(np.float64)).astype(np.float32)
    return hi2, lo2


def _fr(h, l):
    return Fraction(float(h)) + Fraction(float(l))


def test_df64_operations_match_exact_arithmetic():
    rng = np.random.default_rng(5)
    n = 400
    a = _words(rng, n)
    b = _words(rng, n)
    c = _words(rng, n)
    # a share of near-cancelling sums and products, where a careless adder fails
    b[0][:50], b[1][:50] = -a[0][:50], (-a[1][:50] * 0.5).astype(np.float32)
    c[0][50:100] = (-(a[0][50:100].astype(np.float64) * b[0][50:100])).astype(np.float32)
    c[1][50:100] = 0.0   # keep (hi, lo) normalised after replacing hi
    with tempfile.TemporaryDirectory() as td:
        exe = os.path.join(td, "df64_check")
        r = subprocess.run([_compiler(), "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC,
                            os.path.join(HERE, "native", "df64_check.cpp"), "-o", exe], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        lines = "\n".join(" ".join(float(v).hex() for v in (a[0][i], a[1][i], b[0][i], b[1][i], c[0][i], c[1][i]))
                          for i in range(n))
        res = subprocess.run([exe], input=lines, capture_output=True, text=True, check=True).stdout.split("\n")
    u2 = Fraction(1, 2 ** 48)
    for i in range(n):
        w = [float.fromhex(t) for t in res[i].split()]
        got = [_fr(w[2 * k], w[2 * k + 1]) for k in range(8)]
        A, B, Cc = _fr(a[0][i], a[1][i]), _fr(b[0][i], b[1][i]), _fr(c[0][i], c[1][i])
        exact = [A + B, A - B, A * B, A / B]
        for k, e in enumerate(exact):
            assert abs(got[k] - e) <= 8 * u2 * abs(e), (i, k, float(got[k]), float(e))
        # sqrt: compare squares (relative error doubles)
        assert abs(got[4] * got[4] - abs(A)) <= 16 * u2 * abs(A), (i, "sqrt")
        # fma with the sloppy adder: error bounded by the summands' magnitudes
        e = A * B + Cc
        assert abs(got[5] - e) <= 16 * u2 * (abs(A * B) + abs(Cc)), (i, "fma")
        # the fused two-product forms: error bounded by the magnitudes of their terms
        e = A * B + Cc * A
        assert abs(got[6] - e) <= 16 * u2 * (abs(A * B) + abs(Cc * A)), (i, "dot2")
        e = Cc + A * B + B * Cc
        assert abs(got[7] - e) <= 16 * u2 * (abs(Cc) + abs(A * B) + abs(B * Cc)), (i, "fma2")
        # every result is normalised: |lo| <= ulp(hi) / 2
        for k in range(8):
            hi, lo = w[2 * k], w[2 * k + 1]
            if hi != 0.0:
                assert abs(lo) <= np.spacing(np.float32(abs(hi))) / 2 * 1.0000001, (i, k, hi, lo)
