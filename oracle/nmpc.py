"""FP64 oracle of the feedback NMPC loop of §IV-C, run against a simulated plant.

TEST INFRASTRUCTURE: only the tests use this module. It strings together the oracle's pinned
parts (rollouts, MPPI weights and update, least-squares Jacobians, TVLQR) in the order §IV-C
gives; it shares nothing with the CUDA library. A closed loop has no closed form; the loop is
pinned through the cases that reduce to its pinned parts (the plant equal to the model, no
latency, a vanishing MPPI temperature, the projection recomputed as a policy rollout from each
replan's snapshot, the schedule by hand). The tracking instance's wake under an unknown
disturbance is checked only against its definition restated.

The loop, as read from §IV-C (N steps of a fixed-length manoeuvre, controls u = phidot):
  * a tracking instance of the model follows the plant: at every control step its glider state
    is replaced by the observed one and it is stepped with the applied control;
  * every P steps (t > 0, t + L < N) a replan starts from a copy of the tracking instance with
    the observed glider state: the copy is projected L steps ahead under the current
    closed-loop policy (the replanning time), then MPPI (`iterations` reweightings of K
    rollouts over the remaining N - t - L steps, warm-started from the previous nominal
    controls) and the least-squares / TVLQR synthesis around the new nominal run from it;
  * the new policy takes effect at step t + L (at once when L = 0), before the replan due at
    that step (when L = P) starts, so that replan projects under it; the control at step t is
    ubar_t - H_t (x_t - xbar_t) of the policy in effect. L <= P: with a longer latency a plan
    would be replaced before it took effect.
Random draws are inputs: per plan p, noise[p] = (eps (iterations, K, N) binary32 MPPI
perturbations, xi (K, 7) initial-state perturbations, zeta (K, N) binary32 control
perturbations of the synthesis rollouts); plan p uses the first H_r columns.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import State, mppi_update, mppi_weights, rollout, terminal_cost
from . import policy as P


@dataclass
class Config:
    horizon: int            # N
    replan_every: int       # P
    latency: int            # L
    rollouts: int           # K (MPPI and synthesis)
    iterations: int
    lam: float
    qc: tuple
    qf: tuple
    rc: float


@dataclass
class Policy:
    t0: int                 # first step the policy covers
    ubar: np.ndarray        # (N,) absolute-time nominal controls (binary32 values)
    xbar: np.ndarray        # (N - t0 + 1, 7)
    gains: np.ndarray       # (N - t0, 7)

    def control(self, t: int, x) -> float:
        j = t - self.t0
        return float(self.ubar[t]) - float(self.gains[j] @ (np.asarray(x) - self.xbar[j]))


def _f32(a):
    return np.asarray(a, np.float64).astype(np.float32).astype(np.float64)


def plan(cfg: Config, params: dict, snap: State, mu, t0: int, noise) -> tuple:
    """MPPI from the snapshot over steps t0..N-1, then the policy synthesis around the result.
    Returns (mu (N,), Policy)."""
    eps, xi, zeta = noise
    Hr = cfg.horizon - t0
    parts = snap.particles
    mu = np.array(mu, np.float64)
    kw = dict(capacity=snap.capacity, gb_prev=snap.gb_prev, glev_prev=snap.glev_prev,
              has_prev=snap.has_prev, n_dist=snap.n_dist)
    for it in range(cfg.iterations):
        ctrl = _f32(mu[None, t0:] + eps[it][:, :Hr].astype(np.float64))
        J = np.array([rollout(params, parts, snap.xg, ctrl[i], **kw)["cost"] for i in range(cfg.rollouts)])
        w = mppi_weights(_f32(J), cfg.lam)
        mu[t0:] = _f32(mppi_update(_f32(w), ctrl))
    nom = rollout(params, parts, snap.xg, mu[t0:], want_traj=True, **kw)
    xbar = np.vstack([snap.xg, nom["traj"]])
    x0 = xbar[0][None, :] + np.asarray(xi, np.float64)
    u = _f32(mu[None, t0:] + zeta[:, :Hr].astype(np.float64))
    traj = np.stack([rollout(params, parts, x0[i], u[i], want_traj=True, **kw)["traj"]
                     for i in range(cfg.rollouts)])
    A, B = P.ls_jacobians(x0, traj, u, xbar, mu[t0:], params["dt"])
    gains, _ = P.tvlqr(A, B, params["dt"], cfg.qc, cfg.qf, cfg.rc)
    return mu, Policy(t0, mu.copy(), xbar, gains)


def run(cfg: Config, params: dict, parts, x0, mu0, noise, capacity: int, pair=None,
        compensate: bool = False):
    """Closed loop against a plant model (the same model). With `pair` = (x1, z1, g1, x2, z2,
    g2) the plant's wake holds that disturbance pair from the start; with `compensate` the
    tracking instance holds it too, so the planner knows of it. Returns dict(x (N + 1, 7) plant
    states, u (N,) applied controls, cost, plans (list of t0), policies (the plans' Policy
    objects, in the same order), snapshots (for each replan after the first, the tracking
    instance's copy with the observed glider state, before its projection))."""
    N, Pn, L = cfg.horizon, cfg.replan_every, cfg.latency
    if L > Pn:
        raise ValueError("the latency must not exceed the replanning period")
    tracking = State(params, parts, x0, capacity)
    plant = State(params, parts, x0, capacity)
    if pair is not None:
        plant.inject_pair(*pair)
        if compensate:
            tracking.inject_pair(*pair)
    mu, pol = plan(cfg, params, tracking.copy(), mu0, 0, noise[0])
    plans, policies, snapshots, pending, used = [0], [pol], [], None, 1
    xs, us = [plant.xg.copy()], []
    for t in range(N):
        x_obs = plant.xg.copy()
        if pending is not None and t == pending.t0:
            pol, pending = pending, None
        if t > 0 and t % Pn == 0 and t + L < N and used < len(noise):
            snap = tracking.copy()
            snap.xg[:] = x_obs
            snapshots.append(snap.copy())
            for k in range(L):
                snap.step(pol.control(t + k, snap.xg))
            mu, pending = plan(cfg, params, snap, mu, t + L, noise[used])
            used += 1
            plans.append(t + L)
            policies.append(pending)
            if L == 0:
                pol, pending = pending, None
        u = pol.control(t, x_obs)
        tracking.xg[:] = x_obs
        tracking.step(u)
        plant.step(u)
        us.append(u)
        xs.append(plant.xg.copy())
    return dict(x=np.array(xs), u=np.array(us), cost=terminal_cost(params, plant.xg), plans=plans,
                policies=policies, snapshots=snapshots)
