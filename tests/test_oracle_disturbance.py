"""Pins of the disturbance pair (§V): convected with the wake, left out of merging, and removed
at the first step whose end state has the pair's segment crossing the chord line offset by
2 % of the chord against the normal. The crossing is decided here by solving for the
intersection parameters of the two segments, independently of the oracle's orientation test,
and the chord from the plate's placement (centre x_w = x_g - l_w (cos, sin) theta, leading edge
at + c/2 (cos, sin) theta, normal (-sin, cos) theta)."""
import math

import numpy as np
import pytest

import workloads as W


def _offset_chord(p, xg):
    th = xg[2]
    c, s = math.cos(th), math.sin(th)
    xw = np.array([xg[0] - p["l_w"] * c, xg[1] - p["l_w"] * s])
    half = 0.5 * p["chord"] * np.array([c, s])
    off = -0.02 * p["chord"] * np.array([-s, c])
    return xw + half + off, xw - half + off


def _crosses(p0, p1, a, b):
    M = np.column_stack([p1 - p0, -(b - a)])
    if abs(np.linalg.det(M)) < 1e-14:
        return False
    s, t = np.linalg.solve(M, a - p0)
    return 0.0 < s < 1.0 and 0.0 < t < 1.0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pair_removed_at_first_crossing(ora, seed):
    p = W.fixed_plate_params()
    pair, xg, cap = W.fixed_plate_initial(seed)
    a = ora.State(p, np.zeros((0, 3)), xg, cap)
    a.inject_pair(*pair[0], *pair[1])
    b = a.copy()
    b.n_dist = 0                           # the same particles, never terminated
    first = None
    for k in range(200):
        a.step(0.0)
        b.step(0.0)
        P = b.particles
        hit = _crosses(P[0, :2], P[1, :2], *_offset_chord(p, b.xg))
        if hit:
            first = k
            assert a.n_dist == 0 and a.n == b.n - 2
            assert np.array_equal(a.particles, b.particles[2:])
            assert abs(a.g[:a.n].sum() - (b.g[:b.n].sum() - P[0, 2] - P[1, 2])) < 1e-12
            break
        assert a.n_dist == 2 and np.array_equal(a.particles, b.particles), k
    assert first is not None and first > 50      # the pair travels ~2c before it reaches the plate


def test_pair_left_out_of_merging(ora):
    p = dict(W.glider_params(), n_wake_max=10, gamma_decay=0.5)
    s = ora.State(p, W.background_field(5, 8), W.GLIDER_X0, 14)
    s.inject_pair(50.0, 0.0, 0.3, 50.0, 1.0, -0.3)      # far from the plate: never crosses
    decay = math.exp(-0.5 * p["dt"])
    for k in range(1, 16):
        s.step(0.0)
        assert s.n_dist == 2 and s.n == min(2 + 8 + 2 * k, 12)
        assert s.g[0] == pytest.approx(0.3 * decay ** k, rel=1e-12)
        assert s.g[1] == pytest.approx(-0.3 * decay ** k, rel=1e-12)
