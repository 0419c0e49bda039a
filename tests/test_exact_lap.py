"""The exact integer sum of the Laplacian's numerator (csrc/exact_lap.h), the
arithmetic of the FP64 defect kernels, checked on the CPU against exact
rational arithmetic: S = sum_k u_k - N u_p is the correctly rounded exact
value whenever every value lies within 5 binades of the largest, and within
half an ulp of S plus N + 1 units of 2^(E - 1080) otherwise (E the largest
biased exponent); a zero sum is +0.0, and non-finite inputs and a nonzero
sum of tiny values hand back to FP64.
"""
import ctypes as C
import math
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1111_0983_gb300", "csrc")


@pytest.fixture(scope="module")
def lap(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ is missing")
    so = str(tmp_path_factory.mktemp("exl") / "exact_lap_check.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC,
                    os.path.join(ROOT, "tests", "exact_lap_check.cpp"), "-o", so], check=True)
    L = C.CDLL(so)
    L.exl_lap.restype = C.c_int
    L.exl_lap.argtypes = [C.c_int, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]

    def call(up, nb):
        arr = (C.c_double * len(nb))(*nb)
        out = C.c_double(math.nan)
        ok = L.exl_lap(len(nb), up, arr, C.byref(out))
        return ok, out.value
    return call


def exact(up, nb):
    return sum(Fraction(x) for x in nb) - len(nb) * Fraction(up)


def biased(x):
    return max(1, (np.float64(x).view(np.uint64) >> np.uint64(52)).item() & 0x7ff)


def check_case(lap, up, nb):
    ok, s = lap(up, nb)
    assert ok == 1, (up, nb)
    ex = exact(up, nb)
    vals = [up] + list(nb)
    E = max(biased(x) for x in vals)
    if all(E - biased(x) <= 5 or x == 0.0 for x in vals):
        assert s == float(ex), (up, nb, s, float(ex))   # correctly rounded
    else:
        bound = Fraction(math.ulp(s)) / 2 + (len(nb) + 1) * Fraction(2) ** (E - 1080)
        assert abs(Fraction(s) - ex) <= bound, (up, nb, s, float(ex))


@pytest.mark.parametrize("n", [4, 6])
def test_smooth_neighbourhoods_are_correctly_rounded(lap, n):
    """Values of a smooth function at a node and its neighbours (the case of
    every converged solve): the result equals the exact sum rounded once."""
    rng = np.random.default_rng(11)
    for _ in range(4000):
        c = rng.uniform(-2, 2) * 10.0 ** rng.integers(-8, 3)
        h = 2.0 ** -rng.integers(6, 12)
        g = rng.uniform(-1, 1, n) * abs(c) * h
        q = rng.uniform(-1, 1, n) * abs(c) * h * h
        check_case(lap, c, [float(c + a + b) for a, b in zip(g, q)])


@pytest.mark.parametrize("n", [4, 6])
def test_mixed_magnitudes_signs_zeros_and_denormals(lap, n):
    """Sign changes, zeros (nodes off the domain read as 0), values many
    binades apart (truncated, within the stated bound) and denormals."""
    rng = np.random.default_rng(12)
    pool = [0.0, -0.0, 5e-324, -2.5e-310, 1e-300, 1.0, -1.0, 3.0, 2.0 ** 60, -(2.0 ** -40), 0.1, -7.25]
    for _ in range(4000):
        vals = [pool[i] if rng.random() < 0.3 else float(rng.uniform(-1, 1) * 10.0 ** rng.integers(-30, 30))
                for i in rng.integers(0, len(pool), n + 1)]
        ok, _ = lap(vals[0], vals[1:])
        if ok == 0:
            # only a nonzero sum of values below 2^-1015 hands back
            assert max(abs(v) for v in vals) < 2.0 ** -1014 and exact(vals[0], vals[1:]) != 0
            continue
        check_case(lap, vals[0], vals[1:])


def test_cancellation_and_extremes(lap):
    # exact cancellation to zero, the largest finite doubles, a difference that FP64
    # summation of the values (not of differences) would lose
    check_case(lap, 1.0, [1.0, 1.0, 1.0, 1.0])
    assert lap(1.0, [1.0] * 6)[1] == 0.0
    big = np.finfo(np.float64).max
    check_case(lap, big / 8, [big / 8] * 5 + [-big / 8])
    x = 1.0 + 2.0 ** -52
    check_case(lap, x, [1.0, x, x, x + 2.0 ** -51])
    assert lap(1.0, [1.0, 1.0, 1.0, 1.0 + 2.0 ** -52])[1] == 2.0 ** -52


def test_non_finite_and_tiny_values_hand_back(lap):
    for bad in (math.inf, -math.inf, math.nan):
        assert lap(1.0, [1.0, bad, 0.0, 2.0])[0] == 0
        assert lap(bad, [1.0, 1.0, 0.0, 2.0])[0] == 0
    assert lap(1e-310, [0.0, 1e-310, -1e-309, 0.0])[0] == 0
    # a zero sum is exact at any size, the all-zero start of a solve included
    assert lap(0.0, [0.0, 0.0, 0.0, 0.0]) == (1, 0.0)
    assert lap(1e-310, [1e-310] * 6) == (1, 0.0)
