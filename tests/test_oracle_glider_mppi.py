"""Pins of the oracle's glider dynamics (§III-B, Eqs. 18-22), terminal cost (Eq. 24) and
MPPI reweighting (Eq. 25)."""
import math

import numpy as np
import pytest

import workloads as W


def test_ballistic_euler_recurrence(ora):
    """With rho = 0 there is no wing or elevator load: explicit Euler gives
    xdot const, zdot_n = zdot_0 - n g dt, z_n = z_0 + n dt zdot_0 - g dt^2 n(n-1)/2,
    theta_n = theta_0 + n dt thetadot, phi_n = phi_0 + dt sum u."""
    p = dict(W.glider_params(), rho=0.0)
    xg0 = np.array([0.2, 1.0, 0.1, 0.05, 7.0, 0.5, 0.3])
    u = np.linspace(-2, 3, 60)
    out = ora.rollout(p, np.zeros((0, 3)), xg0, u, want_traj=True)
    n, dt, g = len(u), p["dt"], p["g"]
    ref = np.array([
        0.2 + n * dt * 7.0,
        1.0 + n * dt * 0.5 - g * dt * dt * n * (n - 1) / 2,
        0.1 + n * dt * 0.3,
        0.05 + dt * u.sum(),
        7.0, 0.5 - n * g * dt, 0.3])
    assert np.allclose(out["xg"], ref, rtol=1e-12, atol=1e-12)


def test_wing_velocity_is_derivative_of_wing_position(ora):
    """Eq. 18's wing velocity is the time derivative of its wing position along any path."""
    p = W.glider_params()
    def state(t):
        return np.array([1 + 2 * t + t * t, -0.5 * t ** 3, 0.4 * math.sin(3 * t), 0.0,
                         2 + 2 * t, -1.5 * t * t, 1.2 * math.cos(3 * t)])
    h = 1e-5
    for t in (0.1, 0.7, 1.3):
        fd = (ora.plate_geometry(p, state(t + h))["xw"] - ora.plate_geometry(p, state(t - h))["xw"]) / (2 * h)
        g = ora.plate_geometry(p, state(t))
        assert np.allclose(g["v"], fd, rtol=1e-8, atol=1e-9)
        assert g["omega"] == pytest.approx(state(t)[6])


def test_elevator_unloaded_at_zero_incidence(ora):
    """Choose body rates so that the elevator moves along its own chord (alpha_e = 0,
    Eq. 19): the elevator force (Eq. 20) vanishes and only gravity and the wing act."""
    p = W.glider_params()
    th, ph, thd, u, V = 0.3, -0.2, 0.8, 1.7, 5.0
    a = th + ph
    xd = V * math.cos(a) - p["l"] * thd * math.sin(th) - p["l_e"] * (thd + u) * math.sin(a)
    zd = V * math.sin(a) + p["l"] * thd * math.cos(th) + p["l_e"] * (thd + u) * math.cos(a)
    xg = np.array([0, 0, th, ph, xd, zd, thd])
    f = ora.glider_rhs(p, xg, (0.0, 0.0), 0.0, u)
    assert f[4] == pytest.approx(0.0, abs=1e-12)
    assert f[5] == pytest.approx(-p["g"], rel=1e-12)
    assert f[6] == pytest.approx(0.0, abs=1e-12)
    fw = np.array([3.0, -2.0])
    f = ora.glider_rhs(p, xg, fw, 0.5, u)
    arm = -p["l_w"] * np.array([math.cos(th), math.sin(th)])
    assert f[4] == pytest.approx(fw[0] / p["mass"], rel=1e-12)
    assert f[6] == pytest.approx((arm[0] * fw[1] - arm[1] * fw[0] + 0.5) / p["inertia"], rel=1e-12)


def test_tail_is_pitch_stabilising(ora):
    """A nose-up elevator incidence lifts the tail and pitches the nose down."""
    p = W.glider_params()
    xg = np.array([0, 0, 0.0, 0.1, 7.0, 0.0, 0.0])
    f = ora.glider_rhs(p, xg, (0.0, 0.0), 0.0, 0.0)
    assert f[6] < 0 and f[5] > -p["g"]


def test_terminal_cost(ora):
    p = W.glider_params()
    xd = np.array(p["x_d"])
    assert ora.terminal_cost(p, xd) == 0.0
    e = np.eye(7)
    for k in range(7):
        assert ora.terminal_cost(p, xd + 2.0 * e[k]) == pytest.approx(4.0 * p["q"][k])


def test_mppi_weights_properties(ora):
    J = W.costs_synthetic(0, 256).astype(np.float64)
    for lam in (1.0, 10.0, 100.0):
        w = ora.mppi_weights(J, lam)
        assert w.sum() == pytest.approx(1.0, abs=1e-14)
        assert w.argmax() == J.argmin()
        assert np.all(np.diff(w[np.argsort(J)]) <= 1e-18)
        # shift invariance of J
        assert np.allclose(ora.mppi_weights(J + 123.0, lam), w, rtol=1e-12, atol=1e-300)
    assert np.allclose(ora.mppi_weights(J, 1e12), np.full(len(J), 1 / len(J)), rtol=1e-9)
    w0 = ora.mppi_weights(J, 1e-6)
    assert w0[J.argmin()] == pytest.approx(1.0) and w0.sum() == pytest.approx(1.0)


def test_mppi_two_sample_closed_form(ora):
    J = np.array([3.0, 5.5])
    lam = 2.0
    w = ora.mppi_weights(J, lam)
    assert w[0] == pytest.approx(1.0 / (1.0 + math.exp(-(J[1] - J[0]) / lam)), rel=1e-14)


def test_mppi_update_convex_combination(ora):
    rng = np.random.default_rng(0)
    xi = rng.normal(size=(5, 7))
    w = np.array([0.1, 0.2, 0.3, 0.25, 0.15])
    mu = ora.mppi_update(w, xi)
    assert np.allclose(mu, w @ xi, rtol=1e-14)
    same = np.tile(rng.normal(size=7), (5, 1))
    assert np.allclose(ora.mppi_update(w, same), same[0], rtol=1e-14)


def test_rollout_matches_stepping(ora):
    p, field, xg0, eps = W.mppi_c2(0, K=2, H=12, n=100)
    out = ora.rollout(p, field, xg0, eps[0].astype(np.float64), want_traj=True, want_field=True)
    s = ora.State(p, field, xg0, 100 + 24)
    for k in range(12):
        s.step(float(eps[0, k]))
        assert np.array_equal(out["traj"][k], s.xg)
    assert np.array_equal(out["field"], s.particles)
    assert out["cost"] == ora.terminal_cost(p, s.xg)
