"""Pins of the policy oracle (§IV-B): least squares recovers a known linear system exactly
from noiseless data, and the TVLQR recursion agrees with the same finite-horizon LQ problem
solved directly as one quadratic in the stacked controls."""
import numpy as np
import pytest

from oracle import policy as P


def _linear_data(rng, K, H, dt):
    """Trajectories of a known time-varying linear model in the structure of §IV-B, generated
    step by step here (not through the oracle): the kinematic rows integrate the velocities, phi
    integrates u, the accelerations are f_bar + A_hat dx + B_hat du."""
    Ah = rng.normal(0.0, 1.0, (H, 3, 5))
    Bh = rng.normal(0.0, 1.0, (H, 3))
    ubar = rng.normal(0.0, 1.0, H)
    xbar = np.zeros((H + 1, 7))
    xbar[0] = rng.normal(0.0, 1.0, 7)
    fbar = rng.normal(0.0, 1.0, (H, 3))
    for k in range(H):
        d = np.zeros(7)
        d[0:3] = xbar[k, 4:7]
        d[3] = ubar[k]
        d[4:7] = fbar[k]
        xbar[k + 1] = xbar[k] + dt * d
    X = np.zeros((K, H + 1, 7))
    X[:, 0] = xbar[0] + rng.normal(0.0, 0.1, (K, 7))
    U = ubar[None, :] + rng.normal(0.0, 0.3, (K, H))
    for k in range(H):
        dx = X[:, k] - xbar[k]
        du = U[:, k] - ubar[k]
        d = np.zeros((K, 7))
        d[:, 0:3] = X[:, k, 4:7]
        d[:, 3] = U[:, k]
        for r in range(3):
            acc = fbar[k, r] + du * Bh[k, r]
            for c, col in enumerate((2, 3, 4, 5, 6)):
                acc = acc + Ah[k, r, c] * dx[:, col]
            d[:, 4 + r] = acc
        X[:, k + 1] = X[:, k] + dt * d
    return X[:, 0], X[:, 1:], U, xbar, ubar, Ah, Bh


def test_least_squares_recovers_known_linear_system():
    rng = np.random.default_rng(5)
    x0, traj, U, xbar, ubar, Ah, Bh = _linear_data(rng, K=48, H=6, dt=0.01)
    A_est, B_est = P.ls_jacobians(x0, traj, U, xbar, ubar, 0.01)
    assert np.abs(A_est - Ah).max() < 1e-8
    assert np.abs(B_est - Bh).max() < 1e-8


def test_assembled_structure():
    A, B = P.assemble(np.arange(15.0).reshape(3, 5) + 1, np.array([7.0, 8.0, 9.0]))
    assert A[0, 4] == A[1, 5] == A[2, 6] == 1.0 and B[3] == 1.0
    assert not A[3].any() and not A[:, :2].any()
    assert A[4, 2] == 1.0 and A[6, 6] == 15.0 and list(B[4:]) == [7.0, 8.0, 9.0]


@pytest.mark.parametrize("seed", [1, 2])
def test_tvlqr_matches_batch_lq_solution(seed):
    """Dynamic programming against direct optimisation: the finite-horizon LQ problem (stage cost
    x'Q_c x + R_c u^2, terminal x'Q_f x, dynamics x_{k+1} = A_k x_k + B_k u_k) is written as one
    quadratic in the stacked controls and minimised by a linear solve. Its optimal first control
    is -H_0 x_0 for every x_0, and its optimal value is x_0' S_0 x_0."""
    rng = np.random.default_rng(seed)
    H, dt = 25, 0.01
    Ah = rng.normal(0.0, 2.0, (H, 3, 5))
    Bh = rng.normal(0.0, 2.0, (H, 3))
    qc = np.array([0.1, 0.1, 5.0, 0.1, 0.1, 0.1, 5.0])
    qf = np.array([400.0, 400.0, 10.0, 1.0, 1.0, 1.0, 1.0])
    rc = 0.01
    gains, S = P.tvlqr(Ah, Bh, dt, qc, qf, rc)
    # prediction matrices: x_k = F[k] x_0 + G[k] u, u = (u_0 .. u_{H-1})
    F = [np.eye(7)]
    G = [np.zeros((7, H))]
    for k in range(H):
        A = np.eye(7)
        A[0, 4] += dt; A[1, 5] += dt; A[2, 6] += dt
        A[4:7, 2:7] += dt * Ah[k]
        B = np.zeros(7)
        B[3] = dt
        B[4:7] = dt * Bh[k]
        Gk = A @ G[k]
        Gk[:, k] += B
        F.append(A @ F[k])
        G.append(Gk)
    M = rc * np.eye(H)
    N = np.zeros((7, H))
    Pm = np.zeros((7, 7))
    for k in range(H + 1):
        Q = np.diag(qf if k == H else qc)
        M += G[k].T @ Q @ G[k]
        N += F[k].T @ Q @ G[k]
        Pm += F[k].T @ Q @ F[k]
    Kbatch = np.linalg.solve(M, N.T)           # u* = -Kbatch x_0
    S0 = Pm - N @ Kbatch
    assert np.abs(Kbatch[0] - gains[0]).max() <= 1e-9 * np.abs(gains[0]).max()
    assert np.abs(S0 - S[0]).max() <= 1e-9 * np.abs(S[0]).max()
    assert np.abs(S[0] - S[0].T).max() <= 1e-12 * np.abs(S[0]).max()


def test_policy_control_law():
    gains = np.array([[1.0, 2.0, 0, 0, 0, 0, 0]])
    xbar = np.zeros((2, 7))
    assert P.policy_control(gains, xbar, [0.5], np.array([0.1, 0.2, 0, 0, 0, 0, 0]), 0) == pytest.approx(0.0)
