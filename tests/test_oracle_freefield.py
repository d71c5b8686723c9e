"""Pins of the oracle's free-field time stepping (Eq. 16 without a plate; Euler and Heun):
exact discrete recurrences, conserved quantities and convergence orders."""
import math

import numpy as np
import pytest

from tests.independent import core_factor


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_corotating_pair_euler_recurrence(ora, kind):
    """Forward Euler on a symmetric co-rotating pair keeps it symmetric; each step maps the
    separation d -> d sqrt(1 + (omega dt)^2) and the angle -> angle + atan(omega dt), with
    omega = Gamma f(d) / (pi d^2)."""
    G, rc, dt = 0.8, 0.1, 0.01
    d, ang = 0.3, 0.2
    P = np.array([[-d / 2 * math.cos(ang), -d / 2 * math.sin(ang), G],
                  [d / 2 * math.cos(ang), d / 2 * math.sin(ang), G]])
    steps = 500
    out = ora.free_euler(P, kind, rc, dt, steps)
    for _ in range(steps):
        om = G * float(core_factor(kind, d, rc)) / (math.pi * d * d)
        d *= math.sqrt(1 + (om * dt) ** 2)
        ang += math.atan(om * dt)
    ref = np.array([[-d / 2 * math.cos(ang), -d / 2 * math.sin(ang)],
                    [d / 2 * math.cos(ang), d / 2 * math.sin(ang)]])
    assert np.allclose(out[:, :2], ref, rtol=0, atol=1e-11)


def test_opposite_pair_euler_translation(ora):
    """An opposite pair keeps its separation under Euler and moves Gamma f(d)/(2 pi d) dt
    per step."""
    G, d, dt, steps = 0.5, 0.5, 0.01, 300
    P = np.array([[0.0, 0.0, G], [d, 0.0, -G]])
    out = ora.free_euler(P, 2, 0.05, dt, steps)
    speed = G * float(core_factor(2, d, 0.05)) / (2 * math.pi * d)
    assert np.allclose(out[:, 1], speed * dt * steps, rtol=1e-12)
    assert np.allclose(out[:, 0], [0.0, d], atol=1e-13)


def _field(n, seed):
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.uniform(-1, 1, (n, 2)), rng.normal(0, 0.1, (n, 1))], 1)


@pytest.mark.parametrize("stepper", ["free_euler", "free_heun"])
def test_linear_impulse_exact_per_step(ora, stepper):
    """sum_i Gamma_i v_i = 0 because the pairwise kernel is odd, so each Euler step and
    each Heun stage conserves the linear impulse sum Gamma (z, -x) to rounding."""
    P = _field(64, 3)
    imp0 = (P[:, 2:3] * np.stack([P[:, 1], -P[:, 0]], 1)).sum(0)
    out = getattr(ora, stepper)(P, 1, 0.05, 0.01, 50)
    imp1 = (out[:, 2:3] * np.stack([out[:, 1], -out[:, 0]], 1)).sum(0)
    assert np.allclose(imp0, imp1, rtol=0, atol=1e-14)
    assert out[:, 2].sum() == P[:, 2].sum()


def test_angular_impulse_euler_step_identity(ora):
    """Sum Gamma |r|^2 is conserved in continuous time (sum Gamma r.v = 0 because K(dr) is
    perpendicular to dr and odd), so one Euler step changes it by exactly
    dt^2 sum Gamma |v|^2."""
    P = _field(32, 4)
    for dt in (0.02, 0.01, 0.005):
        L0 = (P[:, 2] * (P[:, 0] ** 2 + P[:, 1] ** 2)).sum()
        v = ora.free_velocity(P, 1, 0.1)
        out = ora.free_euler(P, 1, 0.1, dt, 1)
        L1 = (out[:, 2] * (out[:, 0] ** 2 + out[:, 1] ** 2)).sum()
        expected = dt * dt * (P[:, 2] * (v ** 2).sum(1)).sum()
        assert L1 - L0 == pytest.approx(expected, rel=1e-6, abs=1e-16)


def test_heun_second_order(ora):
    """Heun's global error falls by ~4 when dt halves (reference: dt/16)."""
    P = _field(24, 5)
    T = 0.4
    ref = ora.free_heun(P, 1, 0.1, T / 320, 320)
    errs = []
    for steps in (20, 40, 80):
        out = ora.free_heun(P, 1, 0.1, T / steps, steps)
        errs.append(np.abs(out[:, :2] - ref[:, :2]).max())
    assert 3.6 < errs[0] / errs[1] < 4.4
    assert 3.6 < errs[1] / errs[2] < 4.4


def test_velocity_at_skip_matches_free(ora):
    P = _field(50, 6)
    idx = np.array([0, 7, 49])
    v = ora.velocity_at(P, P[idx, :2], 1, 0.05, skip=idx)
    full = ora.free_velocity(P, 1, 0.05)
    assert np.array_equal(v, full[idx])
