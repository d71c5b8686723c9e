"""Pins of the oracle's glider dynamics (§III-B, Eqs. 18-22), terminal cost (Eq. 24) and
MPPI reweighting (Eq. 25)."""
import math

import numpy as np
import pytest

import workloads as W
from tests.independent import cross2, elevator_point, point_velocity, wing_point


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


# Hand-chosen glider states (x, z, theta, phi, xdot, zdot, thetadot) and elevator rates u with
# the elevator at incidence: level flight with a deflected elevator, a climb with pitch rate,
# a dive pitching down, and a slow, steep state with the elevator moving (u != 0).
_ELEVATOR_CASES = [
    ((0.0, 0.0, 0.0, 0.1, 7.0, 0.0, 0.0), 0.0),
    ((1.0, -0.5, 0.25, -0.15, 6.0, 1.5, 0.8), 0.0),
    ((-2.0, 3.0, -0.4, 0.3, 8.0, -3.0, -1.1), 0.0),
    ((0.5, 0.2, 0.9, -0.6, 2.5, -1.0, 0.4), 2.3),
]


def _elevator_force_flat_plate(p, xg, u):
    """Elevator load from flat-plate theory (§III-B, Eqs. 19-20), from the geometry alone: the
    elevator point's velocity by differencing its position, the incidence from the cross
    product of the unit velocity with the elevator chord, and the normal force
    (1/2) rho |v|^2 S_e C_n with C_n = 2 sin(alpha_e) along the body-up elevator normal."""
    v = point_velocity(lambda s: elevator_point(s, p["l"], p["l_e"]), xg, u)
    a = xg[2] + xg[3]
    chord = np.array([math.cos(a), math.sin(a)])
    normal = np.array([-math.sin(a), math.cos(a)])
    sin_alpha = cross2(v / np.linalg.norm(v), chord)
    return 0.5 * p["rho"] * (v @ v) * p["s_e"] * (2.0 * sin_alpha) * normal, v


def test_elevator_force_is_flat_plate_normal_force(ora):
    """With no wing load the translational equations (Eq. 21) carry the elevator force alone:
    m (xddot, zddot + g) must equal the flat-plate normal force at each state. A missing 1/2,
    C_n = sin(alpha_e), a wrong S_e or a wrong incidence sign fails here."""
    p = W.glider_params()
    for xg, u in _ELEVATOR_CASES:
        xg = np.array(xg)
        f = ora.glider_rhs(p, xg, (0.0, 0.0), 0.0, u)
        fe = p["mass"] * np.array([f[4], f[5] + p["g"]])
        ref, _ = _elevator_force_flat_plate(p, xg, u)
        assert np.linalg.norm(ref) > 0.05
        assert np.allclose(fe, ref, rtol=1e-7, atol=1e-9 * np.linalg.norm(ref))
    # level flight at 7 m/s with the elevator 0.1 rad nose-up: |F_e| = rho V^2 S_e sin(0.1)
    xg = np.array(_ELEVATOR_CASES[0][0])
    f = ora.glider_rhs(p, xg, (0.0, 0.0), 0.0, 0.0)
    mag = p["mass"] * math.hypot(f[4], f[5] + p["g"])
    assert mag == pytest.approx(1.2 * 49.0 * 0.1 * math.sin(0.1), rel=1e-12)


def test_elevator_force_dissipates(ora):
    """A flat plate's normal force never drives it: with the elevator fixed to the body
    (u = 0) the force's power on the elevator point is -rho S_e |v|^3 sin^2(alpha_e) <= 0."""
    p = W.glider_params()
    for xg, u in _ELEVATOR_CASES[:3]:
        xg = np.array(xg)
        f = ora.glider_rhs(p, xg, (0.0, 0.0), 0.0, u)
        fe = p["mass"] * np.array([f[4], f[5] + p["g"]])
        _, v = _elevator_force_flat_plate(p, xg, u)
        a = xg[2] + xg[3]
        sin_alpha = cross2(v / np.linalg.norm(v), np.array([math.cos(a), math.sin(a)]))
        power = fe @ v
        assert power < 0
        assert power == pytest.approx(-p["rho"] * p["s_e"] * np.linalg.norm(v) ** 3 * sin_alpha ** 2,
                                      rel=1e-6)


def test_pitch_moment_arms_rigid_body_power(ora):
    """Pitch equation (Eq. 22) with the elevator fixed to the body (u = 0): the power of the wing
    force at x_w, the elevator force at x_e and the couple M_w equals the power of the net force
    at the centre of gravity plus torque times pitch rate, (F_w + F_e) . v_cg + tau thetadot,
    for any loads, if and only if tau is the moment of the forces about the centre of gravity
    with their true points of application. The point velocities come from differencing the
    positions (Eq. 18), not from the oracle's formulas. The torque is also checked directly
    as (x_w - x_cg) x F_w + (x_e - x_cg) x F_e + M_w."""
    p = W.glider_params()
    rng = np.random.default_rng(5)
    for xg, _ in _ELEVATOR_CASES[:3]:
        xg = np.array(xg)
        for _ in range(4):
            fw = rng.normal(scale=20.0, size=2)
            mw = float(rng.normal(scale=3.0))
            f = ora.glider_rhs(p, xg, fw, mw, 0.0)
            f0 = ora.glider_rhs(p, xg, (0.0, 0.0), 0.0, 0.0)
            fe = p["mass"] * np.array([f0[4], f0[5] + p["g"]])        # elevator load alone
            tau = p["inertia"] * f[6]
            vw = point_velocity(lambda s: wing_point(s, p["l_w"]), xg, 0.0)
            ve = point_velocity(lambda s: elevator_point(s, p["l"], p["l_e"]), xg, 0.0)
            vcg = xg[4:6]
            lhs = fw @ vw + fe @ ve + mw * xg[6]
            rhs = (fw + fe) @ vcg + tau * xg[6]
            assert lhs == pytest.approx(rhs, rel=1e-7, abs=1e-7)
            xe = elevator_point(xg, p["l"], p["l_e"]) - xg[:2]
            xw = wing_point(xg, p["l_w"]) - xg[:2]
            assert tau == pytest.approx(cross2(xw, fw) + cross2(xe, fe) + mw, rel=1e-10, abs=1e-12)


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


def test_mppi_weights_exclude_diverged_rollouts(ora):
    """Eq. 25 sends a weight to 0 as its cost grows without bound; a cost that is not finite
    (NaN from a rollout that diverged, or an infinity) gets weight 0, and the other weights are
    those of the finite costs alone, bit for bit. With no finite cost the weights are NaN."""
    J = W.costs_synthetic(3, 64).astype(np.float64)
    bad = [0, 5, 17, 63]
    Jb = J.copy()
    Jb[bad] = [np.nan, np.inf, -np.inf, np.nan]
    keep = np.setdiff1d(np.arange(len(J)), bad)
    for lam in (0.5, 10.0):
        w = ora.mppi_weights(Jb, lam)
        assert np.all(w[bad] == 0.0)
        assert np.array_equal(w[keep], ora.mppi_weights(J[keep], lam))
        assert w.sum() == pytest.approx(1.0, abs=1e-14)
    # a non-finite cost below every finite one does not move J_min
    Jc = np.array([np.nan, 2.0, 3.0, -np.inf])
    assert ora.mppi_weights(Jc, 1.0)[1] == pytest.approx(1.0 / (1.0 + math.exp(-1.0)), rel=1e-14)
    assert np.isnan(ora.mppi_weights(np.array([np.nan, np.inf]), 1.0)).all()


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
    p, field, xg0, eps = W.mppi_batch_inputs(0, K=2, H=12, n=100)
    out = ora.rollout(p, field, xg0, eps[0].astype(np.float64), want_traj=True, want_field=True)
    s = ora.State(p, field, xg0, 100 + 24)
    for k in range(12):
        s.step(float(eps[0, k]))
        assert np.array_equal(out["traj"][k], s.xg)
    assert np.array_equal(out["field"], s.particles)
    assert out["cost"] == ora.terminal_cost(p, s.xg)
