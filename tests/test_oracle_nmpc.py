"""Pins of the closed-loop pieces of the oracle: the tracking-policy rollout of §IV-B and the
feedback NMPC loop of §IV-C (oracle/nmpc.py).

A closed loop has no closed form, so these tests use cases that reduce to something fixed
elsewhere:
  * with zero gains, or with the nominal states equal to the open-loop rollout of the nominal
    controls, the feedback term is exactly zero and the policy rollout is the open-loop rollout
    (itself pinned by the model's own tests);
  * the replanning schedule of §IV-C (a replan every P steps, t > 0, taking effect L steps
    later while t + L < N) written out by hand for a few (N, P, L);
  * when the plant is the model (no disturbance, or a disturbance the planner knows of), the
    projection over the latency is exact: every plan's nominal starts at the plant's state at
    the step the plan takes effect, the plant then stays on that nominal, and the applied
    control is the nominal control, bit for bit;
  * when it differs (a disturbance the planner does not know of), each plan's first nominal
    state is the closed-loop policy rollout, over the latency, from the replan's snapshot of the
    tracking instance with the observed glider state; with no latency it is the observed state;
  * with a vanishing temperature the MPPI weights of Eq. 25 pick one rollout, so each plan's
    controls are the previous plan's controls (the warm start) plus one row of that plan's own
    perturbations, iteration after iteration.
Host only.
"""
import itertools

import numpy as np
import pytest

import workloads as W
from oracle import nmpc as ON
from oracle import policy as OP

RING = (2.5, 0.3, -1.0, 2.5, -0.3, 1.0)


def _params():
    return dict(W.glider_params(), n_wake_max=60)


def _cfg(N, P=10, L=5, K=8, iterations=1, lam=10.0):
    return ON.Config(N, P, L, K, iterations, lam, W.TVLQR_QC, W.TVLQR_QF, W.TVLQR_RC)


def _run(cfg, n_plans=3, pair=None, compensate=False, seed=41):
    noise = W.nmpc_noise(seed, n_plans, cfg.iterations, cfg.rollouts, cfg.horizon)
    return ON.run(cfg, _params(), np.zeros((0, 3)), np.array(W.GLIDER_X0),
                  np.zeros(cfg.horizon), noise, 64, pair=pair, compensate=compensate), noise


def _in_effect(r, t):
    """The policy in effect at step t: the last plan whose first step is at or before t."""
    k = max(i for i, t0 in enumerate(r["plans"]) if t0 <= t)
    return r["policies"][k]


def test_policy_rollout_without_feedback_is_the_open_loop_rollout(ora):
    p = _params()
    field = W.background_field(31, 30)
    H, off, cap = 12, 3, 60
    rng = np.random.default_rng(7)
    ubar = rng.normal(0.0, 2.0, H + off).astype(np.float32).astype(np.float64)
    x0 = np.array(W.GLIDER_X0)
    nominal = ora.rollout(p, field, x0, ubar[off:], capacity=cap, want_traj=True)
    # zero gains: the control is the nominal control whatever the nominal states are
    xbar = rng.normal(0.0, 1.0, (H + off + 1, 7))
    r = OP.rollout_closed_loop(p, field, x0, np.zeros((H + off, 7)), xbar, ubar, off, H, cap)
    assert np.array_equal(r["traj"], nominal["traj"])
    # any gains, nominal states on the open-loop trajectory (aligned with the offset)
    xbar = np.full((H + off + 1, 7), np.nan)
    xbar[off] = x0
    xbar[off + 1:] = nominal["traj"]
    gains = rng.normal(0.0, 0.5, (H + off, 7))
    r = OP.rollout_closed_loop(p, field, x0, gains, xbar, ubar, off, H, cap)
    assert np.array_equal(r["traj"], nominal["traj"])
    assert r["cost"] == nominal["cost"]
    # the same rollout with the feedback acting (nominal states one step late) leaves it
    late = xbar.copy()
    late[off + 1:] = xbar[off:-1]
    r = OP.rollout_closed_loop(p, field, x0, gains, late, ubar, off, H, cap)
    assert np.abs(r["traj"] - nominal["traj"]).max() > 1e-6
    # ... and it is the open-loop rollout of the controls the policy law gives along it
    u = [OP.policy_control(gains, late, ubar, x, off + k)
         for k, x in enumerate(np.vstack([x0, r["traj"][:-1]]))]
    again = ora.rollout(p, field, x0, np.array(u), capacity=cap, want_traj=True)
    assert np.array_equal(again["traj"], r["traj"])


@pytest.mark.parametrize("N,P,L,n_plans,plans", [
    (30, 10, 5, 3, [0, 15, 25]),
    (24, 10, 5, 3, [0, 15]),          # the replan at t = 20 would take effect at 25 >= N
    (25, 10, 5, 3, [0, 15]),          # ... and at 25 = N
    (30, 10, 5, 2, [0, 15]),          # two sets of random draws allow two plans
    (30, 40, 5, 3, [0]),
    (30, 10, 0, 4, [0, 10, 20]),
    (31, 10, 10, 4, [0, 20, 30]),     # t = 10, 20 take effect at 20, 30; t = 30 at 40 >= 31
])
def test_replan_schedule(ora, N, P, L, n_plans, plans):
    r, _ = _run(_cfg(N, P, L, K=4), n_plans=n_plans)
    assert r["plans"] == plans
    assert [pol.t0 for pol in r["policies"]] == plans


def test_latency_longer_than_the_replanning_period_is_rejected(ora):
    with pytest.raises(ValueError):
        _run(_cfg(30, 5, 6, K=4))


@pytest.mark.parametrize("L", [5, 10])
@pytest.mark.parametrize("pair", [None, "compensated"])
def test_plant_equal_to_the_model_follows_each_nominal(ora, L, pair):
    N = 32
    r, _ = _run(_cfg(N, 10, L), pair=RING if pair else None, compensate=pair is not None)
    assert len(r["plans"]) >= 2
    for pol in r["policies"]:
        assert np.array_equal(pol.xbar[0], r["x"][pol.t0])          # the projection is exact
    for t in range(N):
        pol = _in_effect(r, t)
        assert r["u"][t] == pol.ubar[t], t
        assert np.array_equal(r["x"][t + 1], pol.xbar[t + 1 - pol.t0]), t
    # the replans changed the controls, so the equalities above are not those of one plan
    later = r["policies"][1]
    assert np.abs(later.ubar[later.t0:] - r["policies"][0].ubar[later.t0:]).max() > 1e-3


def test_unknown_disturbance_moves_the_plant_off_the_nominal(ora):
    N = 32
    r, _ = _run(_cfg(N, 10, 5), pair=RING)
    ref, _ = _run(_cfg(N, 10, 5))
    assert np.abs(r["x"] - ref["x"]).max() > 1e-3
    # the planner does not know of the pair, so its projections miss the plant
    assert all(np.abs(pol.xbar[0] - r["x"][pol.t0]).max() > 1e-6 for pol in r["policies"][1:])
    # with no latency each plan starts from the observed state and applies its nominal control
    r, _ = _run(_cfg(N, 10, 0), n_plans=4, pair=RING)
    assert r["plans"] == [0, 10, 20, 30]
    for pol in r["policies"]:
        assert np.array_equal(pol.xbar[0], r["x"][pol.t0])
        assert r["u"][pol.t0] == pol.ubar[pol.t0]
        if pol.t0:
            assert r["u"][pol.t0 + 1] != pol.ubar[pol.t0 + 1]        # feedback acts after it


@pytest.mark.parametrize("L", [1, 5, 10])
def test_projection_is_the_policy_rollout_from_the_observed_state(ora, L):
    """Under an unknown disturbance each replan starts from the tracking instance with the
    observed glider state and projects L steps under the policy in effect at that step: the
    plan's first nominal state is where the closed-loop policy rollout (oracle/policy.py) from
    that snapshot ends."""
    N = 32
    r, _ = _run(_cfg(N, 10, L), pair=RING)
    assert len(r["snapshots"]) == len(r["plans"]) - 1 >= 2
    for pol, snap in zip(r["policies"][1:], r["snapshots"]):
        t = pol.t0 - L
        assert np.array_equal(snap.xg, r["x"][t])
        eff = _in_effect(r, t)
        proj = OP.rollout_closed_loop(_params(), snap.particles, snap.xg, eff.gains, eff.xbar,
                                      eff.ubar[eff.t0:], t - eff.t0, L, snap.capacity,
                                      gb_prev=snap.gb_prev, glev_prev=snap.glev_prev,
                                      has_prev=snap.has_prev)
        assert np.array_equal(pol.xbar[0], proj["xg"]), t


def test_tracking_instance_is_the_model_driven_by_the_observations(ora):
    """The definition restated (not an independent pin): the tracking instance is the model
    (without the unknown pair) whose glider state is replaced by the observed one before each
    step and which is stepped with the applied control; each replan's snapshot holds its wake."""
    N = 32
    r, _ = _run(_cfg(N, 10, 5), pair=RING)
    model = ora.State(_params(), np.zeros((0, 3)), W.GLIDER_X0, 64)
    t = 0
    for pol, snap in zip(r["policies"][1:], r["snapshots"]):
        for t in range(t, pol.t0 - 5):
            model.xg[:] = r["x"][t]
            model.step(r["u"][t])
        t = pol.t0 - 5
        assert np.array_equal(snap.particles, model.particles), t
        assert np.array_equal(snap.gb_prev, model.gb_prev) and snap.glev_prev == model.glev_prev


def _f32(a):
    return np.asarray(a, np.float64).astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("iterations", [1, 2])
def test_vanishing_temperature_exposes_the_warm_start(ora, iterations):
    """lambda -> 0: each MPPI iteration keeps one perturbed control sequence, so every plan's
    controls from its first step on are the previous plan's (mu0 for the first) plus one row of
    each of its iterations' perturbations, rounded to binary32 after each addition, and the
    controls before its first step are the previous plan's."""
    N = 30
    cfg = _cfg(N, 10, 5, K=6, iterations=iterations, lam=1e-12)
    r, noise = _run(cfg, pair=RING)
    prev = np.zeros(N)
    for pol, (eps, _, _) in zip(r["policies"], noise):
        t0, Hr = pol.t0, N - pol.t0
        assert np.array_equal(pol.ubar[:t0], prev[:t0])
        found = False
        for ks in itertools.product(range(cfg.rollouts), repeat=iterations):
            mu = prev[t0:].copy()
            for it, k in enumerate(ks):
                mu = _f32(mu + eps[it][k, :Hr].astype(np.float64))
            if np.array_equal(mu, pol.ubar[t0:]):
                found = True
                break
        assert found, t0
        prev = pol.ubar
