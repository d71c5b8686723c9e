"""The free-field accumulators: linear scratch and exact, order-independent sums (host only).

The one-evaluation-per-pair free-field kernels add every partial sum of a particle's velocity
into a fixed-point integer (unit 2^-e) per component, kept as three signed 64-bit digit words of
radix 2^42 that receive plain 64-bit additions (no carry until they are combined). vpm_fixed_sum
runs the same conversion, digit split, word additions and combination on the host; these tests
compare it with the exact sum of the same binary32 values (Python fractions), permute the
order, cross the digit boundaries, load the words with the most additions the kernels make, and
check the exponent's bound. No device is needed.
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
    assert b.value == (48 * n + 64 if n else 0)


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


def test_digit_boundaries_and_the_top_of_the_range():
    """Integers whose 24 significant bits straddle bit 42 or 84 of the 128-bit value, and values
    up to 2^125 units (the exponent leaves |sum| below 2^125), of both signs, sum exactly."""
    e = 0
    vals = []
    for top in (41, 42, 43, 50, 60, 65, 83, 84, 85, 100, 110, 124):
        for s in (1.0, -1.0):
            vals.append(np.float32(s * (2.0 ** top) * 1.4142135))   # 24 bits ending near bit `top`
    v = np.array(vals, dtype=np.float32)
    for perm in range(3):
        p = np.random.default_rng(perm).permutation(len(v))
        for sub in (v[p], v[p][::2], v[p][1::3]):
            s, bad = _fixed_sum(sub, e)
            assert bad == 0
            exact = _exact(sub)
            assert abs(Fraction(s) - exact) <= abs(exact) * Fraction(1, 2 ** 52), (perm, sub)


def test_words_hold_the_most_additions_a_particle_receives():
    """At n = 2^30 particles a particle receives at most n / 1024 + n / 16384 + 3 partial sums.
    That many of the largest values one word can take, all positive (the low word then reaches
    about 2^62 and must not overflow), sum exactly; so does a mixed-sign set of the same count
    that loads the middle and top words, with a total inside the 128-bit range."""
    n = 1 << 30
    count = n // 1024 + n // 16384 + 3
    e = 0
    top0 = np.float32((2.0 ** 24 - 1) * 2.0 ** 18)          # 2^42 - 2^18: bits 18..41, word 0 only
    v = np.full(count, top0, dtype=np.float32)
    s, bad = _fixed_sum(v, e)
    assert bad == 0 and Fraction(s) == Fraction(float(top0)) * count
    rng = np.random.default_rng(5)
    w = (rng.choice([-1.0, 1.0], count) * 2.0 ** rng.integers(60, 105, count) * 1.3).astype(np.float32)
    s, bad = _fixed_sum(w, e)
    exact = _exact(w)
    assert bad == 0 and abs(Fraction(s) - exact) <= abs(exact) * Fraction(1, 2 ** 52)


def test_free_field_rejects_fields_beyond_the_digit_headroom():
    import paper_2509_16079_b300 as V
    L = V.lib()
    st = L.vpm_freefield_velocity(None, (1 << 30) + 1, V.KERNEL_VATISTAS, 0.05, None, None)
    assert st in (V.VPM_ERR_INVALID, V.VPM_ERR_CAPACITY)
