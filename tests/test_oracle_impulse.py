"""Momentum balance of the oracle's plate model (§III-A): the wing load of the unsteady Bernoulli
pressure (Eqs. 13-14) against the force that the rate of change of the vortex impulse of the whole
system gives (bound vortices, the step's shed LEV and TEV, and the wake).

The impulse of a planar vortex system changes only by the force the body exerts on the fluid, so
the fluid's force on the plate is -rho s dP/dt (`tests.independent.vortex_impulse`), evaluated
here by a central difference over the oracle's states. This pins the time-derivative terms of
Eq. 13 from outside the oracle:
  * with only the TEV shed, the derivative of the bound circulations' running sums;
  * with both edges shedding every step, the derivative of the leading-edge circulation. Each step
    sheds a new LEV, whose whole circulation is new over the step. Reading dGamma_LEV/dt as the
    difference of successive LEVs instead gives a normal force of the opposite sign, about 8 times
    too large, and so does dropping the term.
"""
import math

import numpy as np
import pytest

import workloads as W
from tests.independent import vortex_impulse


def _loads_and_impulse_force(ora, p, theta, steps):
    """Normal wing force of Eq. 14 and -rho s dP/dt (central difference; NaN at the ends) per
    step for the fixed plate at incidence theta started impulsively from rest."""
    xg = np.array([0.0, 0.0, theta, 0.0, 0.0, 0.0, 0.0])
    s = ora.State(p, np.zeros((0, 3)), xg, 2 * steps + 4)
    G = ora.plate_geometry(p, xg)
    nb = int(p["n_b"])
    surf = np.vstack([G["b"], G["lev"][None, :], G["tev"][None, :]])   # fixed plate
    P, fn = [], []
    for _ in range(steps):
        wake = s.particles.copy()                  # the wake at the start of the step
        out = s.step(0.0)
        gs = out["gamma_s"]                        # zero for an edge that did not shed
        P.append(vortex_impulse(wake[:, :2], wake[:, 2]) + vortex_impulse(surf, gs[:nb + 2]))
        fn.append(out["fm"][:2] @ G["n"])
    P = np.array(P) * p["rho"] * p["span"]
    f_imp = np.full(steps, np.nan)
    f_imp[1:-1] = (-(P[2:] - P[:-2]) / (2 * p["dt"])) @ G["n"]
    return np.array(fn), f_imp


def test_impulse_sign_convention():
    """An opposite vortex pair moves along its impulse (the helper's sign): lower +1, upper -1 at
    x = 0 move in -x (singular kernel, brute-force velocities)."""
    from tests.independent import biot_savart
    pair = np.array([[0.0, -0.5, 1.0], [0.0, 0.5, -1.0]])
    v = biot_savart(pair, pair[:, :2], 0, 0.0, skip_self=True)
    P = vortex_impulse(pair[:, :2], pair[:, 2])
    assert P[0] < 0 and abs(P[1]) < 1e-15
    assert np.all(v[:, 0] < 0) and np.allclose(v[:, 1], 0.0)


@pytest.mark.parametrize("deg", [3.0, 10.0])
def test_tev_only_load_is_impulse_rate(ora, deg):
    """Trailing edge shedding only (LEV gated off below 20 deg): the Bernoulli load equals the
    impulse force within 5 % over the first half chord of travel (steps 2-49, the impulsive start,
    where the one-step backward differences of Eq. 13 lag the central difference of the impulse)
    and within 2 % over the next 2.5 chords."""
    p = dict(W.fixed_plate_params(), shed_gate=2, alpha_crit=math.radians(20.0))
    fn, fi = _loads_and_impulse_force(ora, p, math.radians(deg), 300)
    assert fn[2:50].mean() == pytest.approx(fi[2:50].mean(), rel=0.05)
    assert fn[50:298].mean() == pytest.approx(fi[50:298].mean(), rel=0.02)


@pytest.mark.parametrize("deg", [10.0, 30.0, 45.0])
def test_lev_shedding_load_follows_impulse(ora, deg):
    """Both edges shed every step (the workloads' setting): over the first half chord of travel
    (steps 2-49) the mean Bernoulli normal force has the impulse force's sign and lies within 25 %
    of it. The remaining difference comes from the discretisation: vortices born 0.02 c from
    the edge collocation points, and a whole LEV formed within each step."""
    p = dict(W.fixed_plate_params(), shed_gate=0)
    fn, fi = _loads_and_impulse_force(ora, p, math.radians(deg), 52)
    a, b = fn[2:50].mean(), fi[2:50].mean()
    assert b > 0 and a > 0
    assert a == pytest.approx(b, rel=0.25)
