"""Closed-loop policy rollouts and the feedback NMPC loop of §IV-C on the GPU against the FP64
oracle. Each side simulates its own plant from its own controls; binary64 models on both sides
keep the closed loops within rounding of each other over these short manoeuvres."""
import numpy as np
import pytest

import workloads as W
from oracle import nmpc as ON
from oracle import policy as OP
from tests.gpu_common import cuda

pytestmark = pytest.mark.gpu


def _policy(H, seed):
    rng = np.random.default_rng(seed)
    gains = rng.normal(0.0, 0.5, (H, 7))
    xbar = np.vstack([W.GLIDER_X0] * (H + 1)) + rng.normal(0.0, 0.05, (H + 1, 7))
    ubar = rng.normal(0.0, 2.0, H).astype(np.float32)
    return gains, xbar, ubar


def test_closed_loop_rollouts_and_advance_match_oracle(ora):
    torch, V = cuda()
    p = dict(W.glider_params(), n_wake_max=60)
    field = W.background_field(31, 40)
    H, off, K = 12, 3, 5
    gains, xbar, ubar = _policy(H + off, 32)
    x0, _ = W.policy_samples(33, K, W.GLIDER_X0, np.zeros(H))
    cap = 62
    st = V.State(p, field, W.GLIDER_X0, cap, V.FP64)
    dg, dx, du = (torch.tensor(a, device="cuda") for a in (gains, xbar, ubar))
    out = st.rollout_policy(K, H, dg, dx, du, off, x0=torch.tensor(x0, device="cuda"), want_traj=True)
    traj = out["traj"].cpu().numpy()
    for i in range(K):
        ref = OP.rollout_closed_loop(p, field, x0[i], gains, xbar, ubar.astype(np.float64), off, H, cap)
        assert np.abs(traj[i] - ref["traj"]).max() <= 1e-9, i
        assert abs(out["costs"][i].item() - ref["cost"]) <= 1e-6 * abs(ref["cost"]) + 1e-6
    # in-place projection of the state itself (the root's glider state)
    st.advance_policy(H, dg, dx, du, off)
    ref = OP.rollout_closed_loop(p, field, np.array(W.GLIDER_X0), gains, xbar, ubar.astype(np.float64), off, H, cap)
    parts, xg, _ = st.read()
    assert np.abs(xg - ref["xg"]).max() <= 1e-9
    assert np.abs(parts[:, :2] - ref["state"].particles[:, :2]).max() <= 1e-9
    st.close()


def _cfg(N, threaded=False, latency=5):
    return dict(horizon=N, replan_every=10, latency=latency, rollouts=16, iterations=2, lam=10.0,
                qc=W.TVLQR_QC, qf=W.TVLQR_QF, rc=W.TVLQR_RC, threaded=threaded)


@pytest.mark.parametrize("pair,latency", [(None, 5), ("uncompensated", 5), ("compensated", 5),
                                          ("uncompensated", 10), ("uncompensated", 0)])
def test_nmpc_synchronous_matches_oracle(ora, pair, latency):
    """latency 10 = the replanning period: each plan takes effect at the step the next replan
    starts and that replan projects under it; latency 0: each plan acts at once."""
    torch, V = cuda()
    p = dict(W.glider_params(), n_wake_max=60)
    N = 40
    c = _cfg(N, latency=latency)
    noise = W.nmpc_noise(41, 4, c["iterations"], c["rollouts"], N)
    field, x0, mu0 = np.zeros((0, 3)), np.array(W.GLIDER_X0), np.zeros(N, np.float32)
    ring = (2.5, 0.3, -1.0, 2.5, -0.3, 1.0) if pair else None
    ref = ON.run(ON.Config(N, 10, latency, 16, 2, 10.0, W.TVLQR_QC, W.TVLQR_QF, W.TVLQR_RC),
                 p, field, x0, mu0.astype(np.float64), noise, 64, pair=ring,
                 compensate=pair == "compensated")
    nm = V.NMPC(p, field, 64, x0, mu0, noise, precision=V.FP64, **c)
    plant = V.State(p, field, x0, 64, V.FP64)
    if ring:
        plant.inject_pair(*ring)
        if pair == "compensated":
            nm.inject_pair(*ring)
    xs, us = [plant.glider()], []
    for t in range(N):
        u = nm.control(t, xs[-1])
        plant.step(u)
        us.append(u)
        xs.append(plant.glider())
    st = nm.stats()
    nm.close()
    plant.close()
    assert st["plans_done"] == len(ref["plans"]) == {0: 4, 5: 4, 10: 3}[latency]
    assert np.abs(np.array(us) - ref["u"]).max() <= 1e-5 * (1.0 + np.abs(ref["u"]).max())
    assert np.abs(np.array(xs) - ref["x"]).max() <= 1e-6


@pytest.mark.parametrize("latency", [5, 10])
def test_nmpc_threaded_matches_synchronous_when_the_planner_keeps_up(latency):
    """With control calls spaced well beyond a plan's time, every plan of the two-thread form
    is ready before its first step: it takes the same snapshot, policy and draws as the
    synchronous form, so the applied controls and the plant agree bit for bit."""
    import time
    torch, V = cuda()
    p = dict(W.glider_params(), n_wake_max=60)
    N = 40
    noise = W.nmpc_noise(43, 4, 2, 16, N)
    x0 = np.array(W.GLIDER_X0)
    ring = (2.5, 0.3, -1.0, 2.5, -0.3, 1.0)
    runs = []
    for threaded in (False, True):
        nm = V.NMPC(p, np.zeros((0, 3)), 64, x0, np.zeros(N, np.float32), noise, precision=V.FP64,
                    **_cfg(N, threaded=threaded, latency=latency))
        plant = V.State(p, np.zeros((0, 3)), x0, 64, V.FP64)
        plant.inject_pair(*ring)
        us = []
        for t in range(N):
            us.append(nm.control(t, plant.glider()))
            plant.step(us[-1])
            if threaded:
                time.sleep(0.05)
        st = nm.stats()
        runs.append((np.array(us), plant.glider(), st))
        nm.close()
        plant.close()
    (u0, x_0, s0), (u1, x_1, s1) = runs
    assert s1["plans_skipped"] == 0 and s1["plans_done"] == s0["plans_done"] >= 3
    assert np.array_equal(u0, u1)
    assert np.array_equal(x_0, x_1)


def test_nmpc_threaded_completes():
    """The two-thread form: planning on its own thread and stream while control continues.
    Timing decides which replans run, so only completion and sanity are checked."""
    torch, V = cuda()
    p = dict(W.glider_params(), n_wake_max=60)
    N = 60
    c = dict(_cfg(N, threaded=True), rollouts=64)
    noise = W.nmpc_noise(42, 6, c["iterations"], c["rollouts"], N)
    x0 = np.array(W.GLIDER_X0)
    nm = V.NMPC(p, np.zeros((0, 3)), 62, x0, np.zeros(N, np.float32), noise, **c)
    plant = V.State(p, np.zeros((0, 3)), x0, 62)
    for t in range(N):
        plant.step(nm.control(t, plant.glider()))
    st = nm.stats()
    t0, g, xb, ub = nm.policy()
    nm.close()
    xg = plant.glider()
    plant.close()
    assert np.isfinite(xg).all() and np.isfinite(g[t0:]).all()
    assert st["plans_done"] + st["plans_skipped"] >= 2 and st["plans_done"] >= 1
