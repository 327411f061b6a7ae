"""CPU checks of the float-float (double-word FP32) arithmetic of the mixed
path, on the host instantiation of the same source.

TwoSum and FastTwoSum must be error-free: hi + lo equals a + b exactly.
Each compound operation must stay within its published double-word error
bound.  Here u = 2^-24, and the bounds are those of Joldes, Muller and
Popescu, "Tight and rigorous error bounds for basic building blocks of
double-word arithmetic", ACM TOMS 44 (2017):
- x + y: 3u^2
- x + b: 2u^2
- x * b: 2u^2
- x * y: 5u^2.  The variant used here drops the lo*lo product, so the
  bound is taken as 6u^2.
- 1/x, by one Newton step on the float-float residual: 4u^2.
- A double rounded to float-float: u^2.

Errors are measured exactly, in rational arithmetic.
"""
import ctypes as C
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
U2 = Fraction(1, 2 ** 48)
N = 3000


@pytest.fixture(scope="module")
def ffl(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("ff") / "libff_host.so")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                    "-Xcompiler", "-fPIC,-ffp-contract=off", "-o", out, os.path.join(ROOT, "tests", "ff_host.cu")],
                   check=True)
    L = C.CDLL(out)
    fp = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
    dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
    L.ff_host_two_sum.argtypes = [C.c_int, fp, fp, fp, fp, C.c_int]
    L.ff_host_of_double.argtypes = [C.c_int, dp, fp, fp]
    L.ff_host_binary.argtypes = [C.c_int, C.c_int, fp, fp, fp, fp, fp, fp]
    return L


def _ff_values(rng, n, spread=8):
    """Random float-float numbers (hi, lo) with |lo| <= ulp(hi)/2, magnitudes over 2^+-spread."""
    x = rng.uniform(1, 2, n) * np.exp2(rng.integers(-spread, spread + 1, n)) * rng.choice([-1.0, 1.0], n)
    x = x * (1 + rng.uniform(-1, 1, n) * 2.0 ** -30)  # bits below FP32's 24
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


def _exact(hi, lo):
    return [Fraction(float(h)) + Fraction(float(l)) for h, l in zip(hi, lo)]


def _max_rel(got_hi, got_lo, ref):
    worst = Fraction(0)
    for h, l, r in zip(got_hi, got_lo, ref):
        if r != 0:
            worst = max(worst, abs(Fraction(float(h)) + Fraction(float(l)) - r) / abs(r))
    return worst


def _binary(L, op, xh, xl, yh, yl):
    hi, lo = np.empty_like(xh), np.empty_like(xh)
    L.ff_host_binary(xh.size, op, xh, xl, yh, yl, hi, lo)
    return hi, lo


@pytest.mark.parametrize("fast", [0, 1])
def test_two_sum_is_error_free(ffl, fast):
    rng = np.random.default_rng(11 + fast)
    a = (rng.standard_normal(N) * np.exp2(rng.integers(-20, 21, N))).astype(np.float32)
    b = (rng.standard_normal(N) * np.exp2(rng.integers(-20, 21, N))).astype(np.float32)
    if fast:  # FastTwoSum needs |a| >= |b|
        swap = np.abs(a) < np.abs(b)
        a[swap], b[swap] = b[swap], a[swap].copy()
    hi, lo = np.empty_like(a), np.empty_like(a)
    ffl.ff_host_two_sum(N, a, b, hi, lo, fast)
    assert np.array_equal(hi, a + b)  # the leading part is the rounded sum
    for i in range(N):
        assert Fraction(float(hi[i])) + Fraction(float(lo[i])) == Fraction(float(a[i])) + Fraction(float(b[i]))


def test_of_double_is_nearest_within_u2(ffl):
    rng = np.random.default_rng(12)
    x = rng.standard_normal(N) * np.exp2(rng.integers(-30, 31, N))
    hi, lo = np.empty(N, np.float32), np.empty(N, np.float32)
    ffl.ff_host_of_double(N, x, hi, lo)
    assert np.array_equal(hi, x.astype(np.float32))
    assert _max_rel(hi, lo, [Fraction(float(v)) for v in x]) <= U2


@pytest.mark.parametrize("op,bound", [(0, 3), (1, 3), (2, 6), (3, 2), (4, 2), (5, 4)])
def test_compound_operations_within_bounds(ffl, op, bound):
    rng = np.random.default_rng(20 + op)
    xh, xl = _ff_values(rng, N)
    if op in (0, 1):
        # half of the pairs nearly cancel: y = -+x (1 + tiny) rounded to float-float
        yh, yl = _ff_values(rng, N)
        k = N // 2
        y = -(xh[:k].astype(np.float64) + xl[:k]) * (1 + rng.uniform(-1, 1, k) * 2.0 ** -12)
        if op == 1:
            y = -y
        yh[:k] = y.astype(np.float32)
        yl[:k] = (y - yh[:k].astype(np.float64)).astype(np.float32)
    elif op in (3, 4):
        yh = _ff_values(rng, N)[0]
        yl = np.zeros(N, np.float32)
    else:
        yh, yl = _ff_values(rng, N)
    hi, lo = _binary(ffl, op, xh, xl, yh, yl)
    X, Y = _exact(xh, xl), _exact(yh, yl)
    ref = {0: [a + b for a, b in zip(X, Y)], 1: [a - b for a, b in zip(X, Y)], 2: [a * b for a, b in zip(X, Y)],
           3: [a + b for a, b in zip(X, Y)], 4: [a * b for a, b in zip(X, Y)], 5: [1 / a for a in X]}[op]
    worst = _max_rel(hi, lo, ref)
    assert worst <= bound * U2, float(worst / U2)
    # the result is itself a normalised pair: |lo| <= ulp(hi) / 2
    assert np.all(np.abs(lo.astype(np.float64)) <= np.spacing(np.abs(hi)).astype(np.float64) / 2)
