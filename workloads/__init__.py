"""Seeded synthetic inputs for the VPM-MPPI workloads.

This module is the only code shared by the FP64 CPU oracle and the CUDA path. It holds
the workload definitions (parameter values, sizes, seeds) and draws random numbers with
numpy's PCG64; it contains none of the vortex-particle or MPPI arithmetic. Every random
number the method consumes (background fields, disturbance offsets, control noise) is
drawn here and handed to both sides as an input array.

Coordinates are (x, z) in chord units, z up; a particle row is (x, z, Gamma).
"""
from __future__ import annotations

import math

import numpy as np

# Kernel identifiers used in parameter dictionaries (both sides map them to their own enums).
KERNEL_SINGULAR = 0
KERNEL_VATISTAS = 1  # regularised kernel of §III-A, Eq. 5 (Leishman / Vatistas n=2)
KERNEL_GAUSSIAN = 2  # Gaussian core, factor 1 - exp(-r^2/delta^2)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def glider_params(**over) -> dict:
    """Open constants of the planar glider (§III-B) chosen for a chord-1 wing.

    The paper takes them from an earlier paper that is not available, so these are the
    values this project fixes. The desired perch state and cost weights are the
    paper's (§IV-A and §V-A).
    """
    p = dict(
        n_b=8, chord=1.0, span=1.0, rho=1.2,
        wake_kernel=KERNEL_VATISTAS, r_core=0.05,
        shed_offset=0.02,            # 2 % of the chord (§III-A)
        gamma_decay=0.1,             # 1/s, 0 < gamma < 1 (§III-A)
        shed_gate=0, alpha_crit=math.radians(15.0),
        n_wake_max=0,                # 0: merging off
        u_inf=(0.0, 0.0), dt=0.01, fixed_plate=0,
        mass=5.0, inertia=1.0, g=9.81, l=1.5, l_w=0.3, l_e=0.1, s_e=0.1,
        q=(10.0, 10.0, 1.0, 0.0, 0.2, 0.2, 0.2),
        x_d=(3.5, 0.0, math.pi / 4, 0.0, 0.5, -0.5, 0.0),
    )
    p.update(over)
    return p


GLIDER_X0 = (0.0, 0.0, 0.0, 0.0, 7.0, 0.0, 0.0)  # initial glider state, §IV-A


# --------------------------------------------------------------------------- fixed plate
def fixed_plate_params() -> dict:
    """Fixed flat plate at 45 degrees incidence in a uniform stream of speed 1.

    The plate is held at theta = 45 deg with its centre at the origin and the stream
    flows in -x, so the leading edge is the upper-right end and the incidence is +45 deg.
    Gaussian core delta = 0.05 c, no decay, shedding every step.
    """
    return glider_params(
        wake_kernel=KERNEL_GAUSSIAN, r_core=0.05, gamma_decay=0.0, u_inf=(-1.0, 0.0),
        fixed_plate=1, l_w=0.0,
    )


def fixed_plate_initial(seed: int, steps: int = 200):
    """Disturbance pair of the fixed-plate case and the fixed plate's glider state.

    Two opposite vortices of strength 0.5 spaced 0.5 c apart are centred 2 c upstream
    (+x, since the stream flows in -x) with a vertical offset uniform in +-0.2 c. The
    lower one has +0.5 and the upper -0.5, so the pair's own induction carries it
    toward the plate along with the stream.
    Returns (particles[n,3], glider[7], capacity).
    """
    off = _rng(seed).uniform(-0.2, 0.2)
    parts = np.array([[2.0, off - 0.25, 0.5], [2.0, off + 0.25, -0.5]], dtype=np.float64)
    glider = np.array([0.0, 0.0, math.pi / 4, 0.0, 0.0, 0.0, 0.0])
    return parts, glider, 2 + 2 * steps


# --------------------------------------------------------------------------- MPPI batch
BOX = (-1.0, 5.0, -1.5, 1.5)  # x0, x1, z0, z1: the 6c x 3c background box


def background_field(seed: int, n: int, box=BOX, gamma_std: float = 0.01) -> np.ndarray:
    """n particles uniform in `box` with Gamma ~ N(0, gamma_std^2); rows (x, z, Gamma)."""
    r = _rng(seed)
    x = r.uniform(box[0], box[1], n)
    z = r.uniform(box[2], box[3], n)
    g = r.normal(0.0, gamma_std, n)
    return np.stack([x, z, g], axis=1)


def lattice_field(seed: int, n: int, box=BOX, gamma_std: float = 0.01, jitter: float = 0.25) -> np.ndarray:
    """n particles on a jittered lattice over `box`: the first n cells of a near-square grid with
    at least n cells, each point moved by up to `jitter` cell widths per axis, so no two particles
    come closer than (1 - 2 jitter) cells; Gamma ~ N(0, gamma_std^2); rows (x, z, Gamma)."""
    r = _rng(seed)
    w, h = box[1] - box[0], box[3] - box[2]
    nx = int(np.ceil(np.sqrt(n * w / h)))
    nz = int(np.ceil(n / nx))
    i = np.arange(n)
    cx, cz = w / nx, h / nz
    x = box[0] + (i % nx + 0.5 + r.uniform(-jitter, jitter, n)) * cx
    z = box[2] + (i // nx + 0.5 + r.uniform(-jitter, jitter, n)) * cz
    g = r.normal(0.0, gamma_std, n)
    return np.stack([x, z, g], axis=1)


def mppi_noise(seed: int, K: int, H: int, sigma: float) -> np.ndarray:
    """Control perturbations eps[K, H] ~ N(0, sigma^2), rounded to float32 once."""
    return _rng(seed).normal(0.0, sigma, (K, H)).astype(np.float32)


MPPI_SIGMA_U = 0.1 / 0.01  # 0.1 rad of elevator deflection per 0.01 s step, as a rate


def mppi_batch_inputs(seed: int = 0, K: int = 1024, H: int = 100, n: int = 1000):
    """MPPI batch of 1000-particle root fields: root field, glider x0 and control noise."""
    p = glider_params()
    field = background_field(seed, n)
    eps = mppi_noise(seed + 1000, K, H, MPPI_SIGMA_U)
    return p, field, np.array(GLIDER_X0), eps


def costs_synthetic(seed: int, K: int, scale: float = 50.0) -> np.ndarray:
    """Synthetic rollout costs (positive, spread like quadratic terminal costs)."""
    r = _rng(seed)
    return (scale * r.chisquare(3, K)).astype(np.float32)


# --------------------------------------------------------------------------- uneven batches
def uneven_counts(seed: int, R: int = 4096, lo: int = 64, hi: int = 8192) -> np.ndarray:
    """Particle counts log-uniform in [lo, hi]."""
    u = _rng(seed).uniform(math.log(lo), math.log(hi), R)
    return np.clip(np.rint(np.exp(u)), lo, hi).astype(np.int64)


# --------------------------------------------------------------------------- large free field
def blob_field(seed: int, n: int, n_blobs: int = 64, sigma: float = 0.1, extent: float = 10.0,
               gamma_std: float = 1e-3) -> np.ndarray:
    """Seeded sum of Gaussian blobs: centres uniform in [0, extent]^2, each particle
    picks a blob uniformly and is displaced by N(0, sigma^2) per axis; Gamma ~ N(0, gamma_std^2)."""
    r = _rng(seed)
    centres = r.uniform(0.0, extent, (n_blobs, 2))
    pick = r.integers(0, n_blobs, n)
    pos = centres[pick] + r.normal(0.0, sigma, (n, 2))
    g = r.normal(0.0, gamma_std, n)
    return np.concatenate([pos, g[:, None]], axis=1)


def sample_indices(seed: int, n: int, m: int) -> np.ndarray:
    """m distinct target indices out of n, sorted."""
    return np.sort(_rng(seed).choice(n, size=min(m, n), replace=False)).astype(np.int64)


# --------------------------------------------------------------------------- serving
def serving_scenarios(seed: int, n_scen: int = 16, n_lo: int = 500, n_hi: int = 5000):
    """Resident field sizes and fields of the serving scenarios (box field + pair)."""
    r = _rng(seed)
    sizes = r.integers(n_lo, n_hi + 1, n_scen)
    fields = []
    for s, n in enumerate(sizes):
        f = background_field(seed * 100 + s, int(n) - 2)
        off = r.uniform(-0.2, 0.2)
        pair = np.array([[4.5, off - 0.25, 0.5], [4.5, off + 0.25, -0.5]])
        fields.append(np.concatenate([f, pair], axis=0))
    return fields


def poisson_arrivals(seed: int, rate_hz: float, duration_s: float, n_streams: int):
    """Arrival times (s) and stream ids of merged Poisson streams, sorted by time."""
    r = _rng(seed)
    ts, ids = [], []
    for s in range(n_streams):
        t = 0.0
        while True:
            t += r.exponential(1.0 / rate_hz)
            if t > duration_s:
                break
            ts.append(t)
            ids.append(s)
    order = np.argsort(ts)
    return np.asarray(ts)[order], np.asarray(ids, dtype=np.int64)[order]


def request_sizes(seed: int, n: int, choices=(256, 1024, 4096)) -> np.ndarray:
    return _rng(seed).choice(np.asarray(choices), n)


# ------------------------------------------------------------------ tracking policy (§IV-B)

# TVLQR weights of the experiments (§V-A): diagonals of Q_c and Q_f, and R_c.
TVLQR_QC = (0.1, 0.1, 5.0, 0.1, 0.1, 0.1, 5.0)
TVLQR_QF = (400.0, 400.0, 10.0, 1.0, 1.0, 1.0, 1.0)
TVLQR_RC = 0.01
# Perturbation scales of the synthesis rollouts (the paper tuned its covariances by sweeps and
# does not print them; these are this build's choice): initial state (x, z, theta, phi, xdot,
# zdot, thetadot) and elevator rate.
POLICY_SIGMA_X = (0.01, 0.01, 0.01, 0.01, 0.05, 0.05, 0.05)
POLICY_SIGMA_U = 1.0


def policy_samples(seed: int, K: int, x0bar, ubar, sigma_x=POLICY_SIGMA_X, sigma_u=POLICY_SIGMA_U):
    """Perturbed initial states x0[K, 7] ~ N(x0bar, diag(sigma_x^2)) (float64) and control
    trajectories u[K, H] ~ N(ubar, sigma_u^2) rounded to float32 once."""
    r = _rng(seed)
    x0 = np.asarray(x0bar, np.float64)[None, :] + r.normal(0.0, 1.0, (K, 7)) * np.asarray(sigma_x)
    ubar = np.asarray(ubar, np.float64)
    u = (ubar[None, :] + r.normal(0.0, sigma_u, (K, len(ubar)))).astype(np.float32)
    return x0, u


def policy_random_data(seed: int, K: int, H: int):
    """Unstructured inputs of the least-squares synthesis (for comparing implementations of a
    pure function): x0 (K, 7), traj (K, H, 7), xbar (H + 1, 7) float64, controls (K, H) and
    ubar (H,) float32."""
    r = _rng(seed)
    return (r.normal(0.0, 1.0, (K, 7)), r.normal(0.0, 1.0, (K, H, 7)),
            r.normal(0.0, 1.0, (K, H)).astype(np.float32), r.normal(0.0, 1.0, (H + 1, 7)),
            r.normal(0.0, 1.0, H).astype(np.float32))


def nmpc_noise(seed: int, n_plans: int, iterations: int, K: int, N: int,
               sigma_mppi: float = MPPI_SIGMA_U, sigma_x=POLICY_SIGMA_X, sigma_u=POLICY_SIGMA_U):
    """Random draws of a closed-loop run, per plan: MPPI perturbations eps (iterations, K, N)
    ~ N(0, sigma_mppi^2) (binary32), synthesis initial-state perturbations xi (K, 7) ~
    N(0, diag(sigma_x^2)) and control perturbations zeta (K, N) ~ N(0, sigma_u^2) (binary32)."""
    r = _rng(seed)
    out = []
    for _ in range(n_plans):
        eps = r.normal(0.0, sigma_mppi, (iterations, K, N)).astype(np.float32)
        xi = r.normal(0.0, 1.0, (K, 7)) * np.asarray(sigma_x)
        zeta = r.normal(0.0, sigma_u, (K, N)).astype(np.float32)
        out.append((eps, xi, zeta))
    return out
