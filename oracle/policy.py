"""FP64 oracle of the local feedback policy of §IV-B (trajectory tracking): least-squares
synthesis of the glider's time-varying Jacobians from perturbed rollouts, and TVLQR gains from
the backward Riccati recursion.

TEST INFRASTRUCTURE: only the tests and the benchmark's CPU-baseline leg use this module. It
uses numpy alone (np.linalg.lstsq for each least-squares problem, plain matrix products for the
recursion) and shares nothing with the CUDA library.

Readings taken where §IV-B is silent or garbled (each is stated again in the design notes):
  * The state derivative of rollout i at step k is the explicit-Euler increment of the model,
    (x_{k+1} - x_k) / dt, which equals f(x_k, u_k) exactly; the nominal derivative likewise.
  * The printed sparsity of A_k puts an identity on the first three columns of the kinematic
    rows; d(x, z, theta)/dt = (xdot, zdot, thetadot) puts it on the velocity columns 4..6. The
    phi row is zero (phidot = u, so its B entry is 1). The unknown block A_hat (3 x 5) maps
    (theta, phi, xdot, zdot, thetadot) to the accelerations (xddot, zddot, thetaddot), and
    B_hat (3 x 1) maps u to them.
  * The Riccati recursion is the discrete one printed in §IV-B, applied to the explicit-Euler
    discretisation A_d = I + dt A_k, B_d = dt B_k of the identified continuous Jacobians, with
    S_N = Q_f and the gain H_k formed from S_{k+1} as in the printed gain equation. The printed
    recursion forms S_{k-1} from S_k and A_k, one index apart from the gain equation; S_k is
    taken from S_{k+1} and A_k, the pairing the gain equation uses.
"""
from __future__ import annotations

import numpy as np

STATE = 7
UNKNOWN_COLS = (2, 3, 4, 5, 6)     # theta, phi, xdot, zdot, thetadot
UNKNOWN_ROWS = (4, 5, 6)           # xddot, zddot, thetaddot


def trajectories(x0, traj):
    """States x^i_k for k = 0..H: the initial states (K, 7) followed by the H states after each
    step (K, H, 7) -> (K, H + 1, 7)."""
    x0 = np.asarray(x0, np.float64)
    traj = np.asarray(traj, np.float64)
    return np.concatenate([x0[:, None, :], traj], axis=1)


def regression(x0, traj, controls, xbar, ubar, dt, k):
    """The least-squares problem of §IV-B at step k: rows (dx^i, du^i) restricted to the
    unknown columns, and the derivative deviations of the accelerations.
    Returns Phi (K, 6) and Y (K, 3)."""
    X = trajectories(x0, traj)
    xbar = np.asarray(xbar, np.float64)
    xdot = (X[:, k + 1] - X[:, k]) / dt
    xbar_dot = (xbar[k + 1] - xbar[k]) / dt
    dx = X[:, k] - xbar[k]
    du = np.asarray(controls, np.float64)[:, k] - float(ubar[k])
    Phi = np.column_stack([dx[:, list(UNKNOWN_COLS)], du])
    Y = (xdot - xbar_dot)[:, list(UNKNOWN_ROWS)]
    return Phi, Y


def ls_jacobians(x0, traj, controls, xbar, ubar, dt):
    """A_hat (H, 3, 5) and B_hat (H, 3) by least squares at every step (np.linalg.lstsq)."""
    H = np.asarray(traj).shape[1]
    Ahat = np.zeros((H, 3, 5))
    Bhat = np.zeros((H, 3))
    for k in range(H):
        Phi, Y = regression(x0, traj, controls, xbar, ubar, dt, k)
        theta, *_ = np.linalg.lstsq(Phi, Y, rcond=None)     # (6, 3)
        Ahat[k] = theta[:5].T
        Bhat[k] = theta[5]
    return Ahat, Bhat


def assemble(Ahat_k, Bhat_k):
    """Continuous Jacobians A_k (7 x 7), B_k (7,) with the known structure of §IV-B."""
    A = np.zeros((STATE, STATE))
    A[0, 4] = A[1, 5] = A[2, 6] = 1.0
    for r, row in enumerate(UNKNOWN_ROWS):
        for c, col in enumerate(UNKNOWN_COLS):
            A[row, col] = Ahat_k[r, c]
    B = np.zeros(STATE)
    B[3] = 1.0
    B[list(UNKNOWN_ROWS)] = Bhat_k
    return A, B


def discretise(A, B, dt):
    """Explicit-Euler discretisation of the continuous Jacobians."""
    return np.eye(STATE) + dt * A, dt * B


def tvlqr(Ahat, Bhat, dt, qc, qf, rc):
    """Backward Riccati recursion of §IV-B from S_N = Q_f. qc, qf: the diagonals of Q_c and Q_f;
    rc: the scalar R_c. Returns gains (H, 7) with u_k = u^d_k - H_k (x_k - x^d_k), and S (H + 1,
    7, 7) with S[N] = Q_f."""
    H = len(Ahat)
    Qc = np.diag(np.asarray(qc, np.float64))
    S = np.zeros((H + 1, STATE, STATE))
    S[H] = np.diag(np.asarray(qf, np.float64))
    gains = np.zeros((H, STATE))
    for k in range(H - 1, -1, -1):
        A, B = discretise(*assemble(Ahat[k], Bhat[k]), dt)
        Sn = S[k + 1]
        denom = rc + B @ Sn @ B
        gains[k] = (B @ Sn @ A) / denom
        S[k] = A.T @ Sn @ A - np.outer(A.T @ Sn @ B, B @ Sn @ A) / denom + Qc
    return gains, S


def policy_control(gains, xbar, ubar, x, k):
    """Control of the tracking policy at step k: u^d_k - H_k (x - x^d_k)."""
    return float(ubar[k]) - float(np.asarray(gains)[k] @ (np.asarray(x, np.float64) - np.asarray(xbar)[k]))


def rollout_closed_loop(params, parts, x0, gains, xbar, ubar, offset, H, capacity=None,
                        controls=None, gb_prev=None, glev_prev=0.0, has_prev=0):
    """One rollout of H steps under the tracking policy: at step k the control is
    ubar_j - H_j . (x_k - xbar_j), j = offset + k (plus controls[k] if given), x_k the rollout's
    own glider state. Returns dict(xg, cost, traj, state) with the final oracle State."""
    from . import State, terminal_cost
    parts = np.asarray(parts, np.float64).reshape(-1, 3)
    cap = capacity if capacity is not None else len(parts) + 2 * H
    s = State(params, parts, x0, cap, gb_prev, glev_prev, has_prev)
    traj = np.zeros((H, STATE))
    for k in range(H):
        j = offset + k
        u = float(ubar[j]) - float(np.asarray(gains[j]) @ (s.xg - np.asarray(xbar[j])))
        if controls is not None:
            u += float(controls[k])
        s.step(u)
        traj[k] = s.xg
    return dict(xg=s.xg.copy(), cost=terminal_cost(params, s.xg), traj=traj, state=s)
