"""Pins of the oracle's plate model (§III-A, Eqs. 6-16): no-through-flow residuals, Kelvin's
theorem, invariance under rigid motions, symmetry, and Wagner's indicial lift response
of unsteady thin-airfoil theory."""
import math

import numpy as np
import pytest

import workloads as W
from tests.independent import biot_savart, wagner_jones


def _geometry(p, xg):
    """Plate points written from the readings (wing centre x_w of Eq. 18, LE forward,
    e_t from LE to TE, collocation points at the panel ends, bound vortices at midpoints)."""
    th = xg[2]
    xw = np.array([xg[0] - p["l_w"] * math.cos(th), xg[1] - p["l_w"] * math.sin(th)])
    et = -np.array([math.cos(th), math.sin(th)])
    en = np.array([-math.sin(th), math.cos(th)])
    nb, c = p["n_b"], p["chord"]
    s_c = -c / 2 + np.arange(nb + 1) * c / nb
    s_b = -c / 2 + (np.arange(nb) + 0.5) * c / nb
    col = xw + s_c[:, None] * et
    bnd = xw + s_b[:, None] * et
    ds = p["shed_offset"] * c
    lev, tev = col[0] - ds * et, col[-1] + ds * et
    if p["fixed_plate"]:
        v, om = np.zeros(2), 0.0
    else:
        v = np.array([xg[4] + p["l_w"] * xg[6] * math.sin(th), xg[5] - p["l_w"] * xg[6] * math.cos(th)])
        om = xg[6]
    return dict(xw=xw, et=et, en=en, col=col, bnd=bnd, lev=lev, tev=tev, v=v, om=om)


def _normal_residual(p, xg, wake, gs, shed_lev=True, shed_tev=True):
    """Relative normal velocity at the collocation points from every vortex after the solve."""
    G = _geometry(p, xg)
    nb = p["n_b"]
    pts = G["col"]
    v = biot_savart(wake, pts, p["wake_kernel"], p["r_core"]) if len(wake) else np.zeros_like(pts)
    v = v + biot_savart(np.c_[G["bnd"], gs[:nb]], pts, 0, 0.0)
    shed = []
    if shed_lev:
        shed.append([*G["lev"], gs[nb]])
    if shed_tev:
        shed.append([*G["tev"], gs[nb + 1]])
    if shed:
        v = v + biot_savart(np.array(shed), pts, p["wake_kernel"], p["r_core"])
    rel = pts - G["xw"]
    rot = G["om"] * np.stack([-rel[:, 1], rel[:, 0]], 1)
    vrel = v + np.asarray(p["u_inf"]) - G["v"] - rot
    return vrel @ G["en"]


def _c2_like(seed=0, n=300):
    p = W.glider_params()
    field = W.background_field(seed, n)
    xg = np.array([0.1, -0.05, 0.12, 0.03, 6.5, -0.8, 0.7])
    return p, field, xg


@pytest.mark.parametrize("kernel", [1, 2])
def test_no_through_flow_and_kelvin(ora, kernel):
    p, field, xg = _c2_like()
    p = dict(p, wake_kernel=kernel)
    s = ora.State(p, field, xg, 400)
    for k in range(6):
        wake = s.particles.copy()
        xg_k = s.xg.copy()
        out = s.step(0.3)
        res = _normal_residual(p, xg_k, wake, out["gamma_s"])
        assert np.abs(res).max() < 1e-10 * max(1.0, np.abs(out["vel"]).max())
        assert out["gamma_s"].sum() + wake[:, 2].sum() == pytest.approx(0.0, abs=1e-12)


def test_rigid_motion_invariance(ora):
    """K n is rotation invariant, so Gamma_S is unchanged by a rigid rotation plus translation
    of the whole scene; the wing load rotates with it and the moment is unchanged."""
    p, field, xg = _c2_like(1)
    a = ora.State(p, field, xg, 400)
    oa = a.step(0.0)
    beta, shift = 0.7, np.array([3.0, -2.0])
    R = np.array([[math.cos(beta), -math.sin(beta)], [math.sin(beta), math.cos(beta)]])
    f2 = field.copy()
    f2[:, :2] = field[:, :2] @ R.T + shift
    xg2 = xg.copy()
    xg2[0:2] = R @ xg[0:2] + shift
    xg2[2] += beta
    xg2[4:6] = R @ xg[4:6]
    b = ora.State(p, f2, xg2, 400)
    ob = b.step(0.0)
    assert np.allclose(oa["gamma_s"], ob["gamma_s"], rtol=1e-10, atol=1e-12)
    assert np.allclose(R @ oa["fm"][:2], ob["fm"][:2], rtol=1e-9, atol=1e-9)
    assert oa["fm"][2] == pytest.approx(ob["fm"][2], rel=1e-9, abs=1e-9)


def test_zero_incidence_no_wake_is_unloaded(ora):
    p = dict(W.fixed_plate_params(), wake_kernel=1)
    s = ora.State(p, np.zeros((0, 3)), np.array([0.0, 0.0, 0.0, 0, 0, 0, 0]), 10)
    out = s.step()
    assert np.abs(out["gamma_s"]).max() < 1e-15
    assert np.abs(out["fm"]).max() < 1e-14


def test_mirror_incidence_antisymmetric(ora):
    p = W.fixed_plate_params()
    ga = ora.State(p, np.zeros((0, 3)), np.array([0, 0, 0.3, 0, 0, 0, 0.0]), 10).step()
    gb = ora.State(p, np.zeros((0, 3)), np.array([0, 0, -0.3, 0, 0, 0, 0.0]), 10).step()
    assert np.allclose(ga["gamma_s"], -gb["gamma_s"], atol=1e-14)


def test_wagner_indicial_lift(ora):
    """Impulsively started flat plate at 3 deg with only the TEV shed (LEV gated off): the
    normal force follows Wagner's function (Jones' fit) toward the thin-airfoil value
    2 pi sin(alpha) q c; the centre of pressure sits ahead of mid-chord (nose-up moment)."""
    deg = 3.0
    p = dict(W.fixed_plate_params(), shed_gate=2, alpha_crit=math.radians(20.0))
    al = math.radians(deg)
    s = ora.State(p, np.zeros((0, 3)), np.array([0, 0, al, 0, 0, 0, 0.0]), 900)
    q = 0.5 * p["rho"] * 1.0 ** 2 * p["chord"] * p["span"]
    cn_thin = 2 * math.pi * math.sin(al)
    en = np.array([-math.sin(al), math.cos(al)])
    checks = {200: None, 400: None, 800: None}
    for k in range(1, 801):
        out = s.step()
        if k in checks:
            fn = out["fm"][:2] @ en
            t = k * p["dt"]
            ratio = fn / q / cn_thin
            assert ratio == pytest.approx(wagner_jones(2 * t / p["chord"]), rel=0.04)
            assert 0.75 < out["fm"][2] / (fn * p["chord"] / 4) < 1.0
    assert s.n == 800


def test_gate_mode1_sheds_nothing_below_alpha_crit(ora):
    p = dict(W.fixed_plate_params(), shed_gate=1, alpha_crit=math.radians(10), wake_kernel=1)
    wake = np.array([[1.5, 0.3, 0.2], [2.0, -0.4, -0.1]])
    xg = np.array([0, 0, math.radians(5), 0, 0, 0, 0.0])
    s = ora.State(p, wake, xg, 10)
    out = s.step()
    assert out["shed"] == 0 and s.n == 2
    res = _normal_residual(p, xg, wake, out["gamma_s"], False, False)
    assert np.abs(res[1:-1]).max() < 1e-12
    assert out["gamma_s"].sum() + wake[:, 2].sum() == pytest.approx(0.0, abs=1e-14)
    s2 = ora.State(p, wake, np.array([0, 0, math.radians(15), 0, 0, 0, 0.0]), 10)
    assert s2.step()["shed"] == 2


def test_gate_mode2_sheds_tev_only(ora):
    p = dict(W.fixed_plate_params(), shed_gate=2, alpha_crit=math.radians(10), wake_kernel=1)
    xg = np.array([0, 0, math.radians(5), 0, 0, 0, 0.0])
    s = ora.State(p, np.zeros((0, 3)), xg, 10)
    out = s.step()
    assert out["shed"] == 1 and out["gamma_s"][p["n_b"]] == 0.0
    res = _normal_residual(p, xg, np.zeros((0, 3)), out["gamma_s"], False, True)
    assert np.abs(res[1:]).max() < 1e-12


def test_merging_keeps_circulation(ora):
    p = dict(W.fixed_plate_params(), n_wake_max=20, wake_kernel=1)
    wake = W.background_field(2, 19)
    wake[:, 0] += 3.0
    s = ora.State(p, wake, np.array([0, 0, 0.4, 0, 0, 0, 0.0]), 40)
    for _ in range(10):
        before = s.particles.copy()
        x0 = before[:2, :2].copy()
        out = s.step()
        assert s.n <= 20
        # decay is off in this configuration: merging moves no circulation
        shed = out["gamma_s"][p["n_b"]:].sum()
        assert s.particles[:, 2].sum() == pytest.approx(before[:, 2].sum() + shed, abs=1e-13)
    assert s.n == 20


def test_merge_position_is_mean(ora):
    p = dict(W.fixed_plate_params(), n_wake_max=3, wake_kernel=1)
    wake = np.array([[10.0, 0.0, 0.1], [12.0, 2.0, 0.2]])
    s = ora.State(p, wake, np.array([0, 0, 0.4, 0, 0, 0, 0.0]), 10)
    out = s.step()
    vel = out["vel"]
    moved = wake[:, :2] + p["dt"] * vel[:2]
    assert s.n == 3
    assert np.allclose(s.particles[0, :2], moved.mean(0), atol=1e-15)
    assert s.particles[0, 2] == pytest.approx(0.3, abs=1e-15)


def test_plate_loads_entry_is_the_steps_own(ora):
    """ora_plate_loads (the loads of Eqs. 13-15 from given circulations and plate velocities,
    which the GPU step test feeds with the kernel's own values) returns exactly the loads the
    oracle's step forms, on first and later steps, with both edges shedding and with gating."""
    for params, seed in ((W.glider_params(), 0), (W.glider_params(shed_gate=2), 1)):
        s = ora.State(params, W.background_field(seed, 200), np.array(W.GLIDER_X0), 260)
        rng = np.random.default_rng(seed)
        for k in range(6):
            xg, gb, hp = s.xg.copy(), s.gb_prev.copy(), s.has_prev
            out = s.step(float(rng.normal(0.0, 3.0)))
            fm = ora.plate_loads(params, xg, out["gamma_s"], gb, hp, out["vtilde"])
            assert np.array_equal(fm, out["fm"]), (seed, k)
            assert k == 0 or np.abs(fm).max() > 0
