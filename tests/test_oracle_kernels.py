"""Pins of the oracle's vortex kernels (§III-A, Eqs. 2-5) against facts fixed by the
mathematics: circulation theorems, divergence-free fields, algebraic identities and an
independent 3-D cross-product brute force."""
import math

import numpy as np
import pytest

from tests.independent import biot_savart, core_factor

KINDS = [0, 1, 2]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("R", [0.01, 0.05, 0.2, 3.0])
def test_circulation_around_circle(ora, kind, R):
    """Stokes: the line integral of v around a circle of radius R centred on a unit vortex
    equals the circulation enclosed, Gamma * f(R), counter-clockwise positive."""
    rc = 0.05
    m = 720
    th = (np.arange(m) + 0.5) * 2 * math.pi / m
    pts = np.stack([R * np.cos(th), R * np.sin(th)], 1)
    v = ora.velocity_at(np.array([[0.0, 0.0, 1.0]]), pts, kind, rc)
    tang = np.stack([-np.sin(th), np.cos(th)], 1)
    circ = (v * tang).sum() * (2 * math.pi * R / m)
    expected = 1.0 if kind == 0 else float(core_factor(kind, R, rc))
    assert circ == pytest.approx(expected, rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("kind", KINDS)
def test_divergence_free(ora, kind):
    rng = np.random.default_rng(0)
    src = np.concatenate([rng.uniform(-1, 1, (5, 2)), rng.normal(0, 1, (5, 1))], 1)
    h = 1e-5
    for p in rng.uniform(-1, 1, (10, 2)):
        pts = np.array([p + [h, 0], p - [h, 0], p + [0, h], p - [0, h]])
        v = ora.velocity_at(src, pts, kind, 0.2)
        div = (v[0, 0] - v[1, 0]) / (2 * h) + (v[2, 1] - v[3, 1]) / (2 * h)
        scale = np.abs(v).max() / 0.05
        assert abs(div) < 1e-5 * scale


def test_vatistas_identity(ora):
    """Eq. 5 times Eq. 4 equals Gamma (-dz, dx) / (2 pi sqrt(rc^4 + r^4))."""
    rng = np.random.default_rng(1)
    rc = 0.05
    for dx, dz in rng.normal(0, 0.1, (50, 2)):
        kx, kz = ora.kernel(1, rc, dx, dz)
        r2 = dx * dx + dz * dz
        s = 1.0 / (2 * math.pi * math.sqrt(rc ** 4 + r2 * r2))
        assert kx == pytest.approx(-dz * s, rel=1e-13)
        assert kz == pytest.approx(dx * s, rel=1e-13)


@pytest.mark.parametrize("kind", [1, 2])
def test_regularised_limits(ora, kind):
    """Far from the core the regularised kernels approach the singular one; at r = 0 they
    vanish (the self term of Eq. 16 is excluded)."""
    k0 = ora.kernel(0, 0.05, 5.0, -2.0)
    k1 = ora.kernel(kind, 0.05, 5.0, -2.0)
    assert k1[0] == pytest.approx(k0[0], rel=1e-8) and k1[1] == pytest.approx(k0[1], rel=1e-8)
    assert ora.kernel(kind, 0.05, 0.0, 0.0) == (0.0, 0.0)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n", [1, 2, 17, 64])
def test_free_velocity_brute_force(ora, kind, n):
    rng = np.random.default_rng(n)
    P = np.concatenate([rng.uniform(-1, 1, (n, 2)), rng.normal(0, 0.3, (n, 1))], 1)
    v = ora.free_velocity(P, kind, 0.1)
    ref = biot_savart(P, P[:, :2], kind, 0.1, skip_self=True)
    assert np.allclose(v, ref, rtol=1e-12, atol=1e-14)


def test_opposite_pair_translates(ora):
    """An equal and opposite pair at separation d translates at Gamma f(d) / (2 pi d),
    perpendicular to the line joining it."""
    for kind, rc in [(0, 0.05), (1, 0.05), (2, 0.05), (1, 0.3)]:
        d, G = 0.5, 0.7
        P = np.array([[0.0, 0.0, G], [d, 0.0, -G]])
        v = ora.free_velocity(P, kind, rc)
        speed = G * float(core_factor(kind, d, rc)) / (2 * math.pi * d)
        assert np.allclose(v[0], v[1], rtol=0, atol=1e-15)
        assert v[0][0] == pytest.approx(0.0, abs=1e-15)
        # vortex 0 (CCW, left) and 1 (CW, right): each is carried +z by the other
        assert v[0][1] == pytest.approx(speed, rel=1e-13)


def test_corotating_pair_rotates(ora):
    """Two equal vortices at separation d orbit their midpoint at Gamma f(d) / (pi d^2)."""
    for kind in KINDS:
        d, G = 0.4, 0.9
        P = np.array([[-d / 2, 0.0, G], [d / 2, 0.0, G]])
        v = ora.free_velocity(P, kind, 0.05)
        omega = G * float(core_factor(kind, d, 0.05)) / (math.pi * d * d)
        # counter-clockwise: the right vortex moves +z, the left one -z
        assert v[1][1] == pytest.approx(omega * d / 2, rel=1e-13)
        assert v[0][1] == pytest.approx(-omega * d / 2, rel=1e-13)
