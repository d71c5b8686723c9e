"""The free-field accumulators: linear scratch and exact, order-independent sums (host only).

The one-evaluation-per-pair free-field kernels add every partial sum of a particle's velocity
into two 128-bit fixed-point integers (unit 2^-e) with 64-bit atomic additions and a carry into
the high word. vpm_fixed_sum runs the same conversion and addition on the host; these tests
compare it with the exact sum of the same binary32 values (Python fractions), permute the
order, force carries between the words, and check the exponent's bound. No device is needed.
"""
import ctypes as C
import math
from fractions import Fraction

import numpy as np
import pytest


def _lib():
    import paper_2509_16079_b300 as V
    return V, V.lib()


def _fixed_sum(vals, e):
    V, L = _lib()
    a = np.ascontiguousarray(vals, dtype=np.float32)
    out, bad = C.c_double(), C.c_int()
    V.check(L.vpm_fixed_sum(a.ctypes.data_as(C.c_void_p), len(a), int(e), C.byref(out), C.byref(bad)))
    return out.value, bad.value


def _exact(vals):
    return sum((Fraction(float(v)) for v in np.asarray(vals, dtype=np.float32)), Fraction(0))


@pytest.mark.parametrize("n", [0, 1, 1000, 1 << 20, 1 << 22])
def test_scratch_is_linear(n):
    V, L = _lib()
    b = C.c_size_t()
    V.check(L.vpm_freefield_scratch_bytes(n, C.byref(b)))
    assert b.value == (32 * n + 64 if n else 0)


def test_sum_is_exact_and_order_independent():
    """Values spanning 40 binades with heavy cancellation: the result is the exact sum rounded
    once, within n/2 units of 2^-e from the values' own rounding to the unit, and every order
    gives the same bits."""
    rng = np.random.default_rng(3)
    v = (rng.standard_normal(4000) * np.exp2(rng.integers(-20, 20, 4000))).astype(np.float32)
    v = np.concatenate([v, -v[:3000]])                     # most of the sum cancels
    e = 80
    s0, bad = _fixed_sum(v, e)
    assert bad == 0
    exact = _exact(v)
    assert abs(Fraction(s0) - exact) <= Fraction(len(v), 2) * Fraction(1, 2 ** e) + abs(exact) * Fraction(1, 2 ** 52)
    for seed in range(5):
        p = np.random.default_rng(seed).permutation(len(v))
        assert _fixed_sum(v[p], e)[0] == s0


def test_carries_between_words_and_negative_totals():
    """Values of 2^62 units and more make the low word wrap many times; a negative total and
    an exact zero come out right."""
    e = 40
    big = np.float32(2.0 ** 22) * np.float32(1.75)         # 1.75 * 2^62 units
    v = np.array([big] * 7 + [-big] * 3 + [np.float32(-1.0)], dtype=np.float32)
    s, _ = _fixed_sum(v, e)
    assert Fraction(s) == _exact(v)
    s, _ = _fixed_sum(-v, e)
    assert Fraction(s) == -_exact(v)
    s, _ = _fixed_sum(np.array([big, -big, 3.0, -3.0], dtype=np.float32), e)
    assert s == 0.0


def test_values_below_the_unit_round_to_nearest():
    e = 10
    unit = 2.0 ** -e
    for x in (0.2 * unit, 0.6 * unit, -0.6 * unit, 1.5 * unit, -2.5 * unit):
        s, _ = _fixed_sum(np.array([x], dtype=np.float32), e)
        xf = float(np.float32(x))
        assert s == math.copysign(math.floor(abs(xf) / unit + 0.5) * unit, xf)


def test_nonfinite_values_are_flagged():
    s, bad = _fixed_sum(np.array([1.0, np.nan, 2.0], dtype=np.float32), 20)
    assert bad == 1 and s == 3.0
    assert _fixed_sum(np.array([np.inf], dtype=np.float32), 20)[1] == 1


@pytest.mark.parametrize("kernel,rc", [(1, 0.05), (1, 1e-3), (2, 0.05), (0, 0.0)])
@pytest.mark.parametrize("n,gmax", [(1, 1.0), (1500, 0.03), (1 << 22, 3e-3), (64, 1e-25)])
def test_exponent_bounds_every_sum(kernel, rc, n, gmax):
    """B = n max|Gamma| kappa bounds every partial and total sum; 2^e B lies in [2^124, 2^125),
    so values fit the 128-bit accumulator with two bits to spare and the unit is B 2^-125."""
    V, L = _lib()
    e = C.c_int()
    V.check(L.vpm_fixed_exponent(C.c_float(gmax), n, kernel, rc, C.byref(e)))
    kappa = 2.0 ** 40 if kernel == 0 else 1.0 / float(np.float32(rc))
    B = n * float(np.float32(gmax)) * kappa
    assert 2.0 ** 124 <= B * 2.0 ** e.value < 2.0 ** 125
    # the largest |r q(r)| of each regularised kernel is below kappa
    r = np.geomspace(1e-6, 1e3, 20001) * max(rc, 1e-30)
    if kernel == 1:
        assert (r / np.sqrt(r ** 4 + rc ** 4)).max() <= 1.0 / rc
    elif kernel == 2:
        assert (-np.expm1(-(r / rc) ** 2) / r).max() <= 1.0 / rc


def test_exponent_of_a_field_without_circulation():
    V, L = _lib()
    e = C.c_int(7)
    V.check(L.vpm_fixed_exponent(C.c_float(0.0), 100, 1, 0.05, C.byref(e)))
    assert e.value == 0
