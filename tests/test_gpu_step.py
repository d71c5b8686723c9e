"""Per-step parity of vpm_step against the FP64 oracle (teacher forcing).

The oracle is run forward; at sampled steps its complete state (wake, glider, previous
circulations) is loaded into a GPU state, and one step is taken on both sides from that
identical state. Compared: relative velocities at the plate (Eq. 12), surface circulations
(Eq. 11), wing loads (Eqs. 14-15), convection velocities of every particle (Eq. 16), and the
advanced state.
"""
import math

import numpy as np
import pytest

import workloads as W
from tests.gpu_common import VEL_TOL, cuda, gpu_state, normwise, oracle_state, snapshot

pytestmark = pytest.mark.gpu


def _cases():
    gl = W.glider_params()
    fp = W.fixed_plate_params()
    return {
        "glider_ungated": (gl, W.background_field(0, 1000), np.array(W.GLIDER_X0), [0, 1, 25, 60, 99]),
        "glider_lev_gated": (dict(gl, shed_gate=2), W.background_field(1, 700), np.array(W.GLIDER_X0), [0, 5, 40]),
        "glider_both_gated": (dict(gl, shed_gate=1, alpha_crit=math.radians(3)), W.background_field(2, 400),
                          np.array(W.GLIDER_X0), [0, 10, 30]),
        "glider_merging": (dict(gl, n_wake_max=450), W.background_field(3, 440), np.array(W.GLIDER_X0), [0, 3, 20]),
        "fixed_plate_gaussian": (fp, *W.fixed_plate_initial(0)[:2], [0, 1, 80, 160, 199]),
        "nb2": (dict(gl, n_b=2), W.background_field(4, 300), np.array(W.GLIDER_X0), [0, 7, 30]),
        "nb32": (dict(gl, n_b=32), W.background_field(5, 300), np.array(W.GLIDER_X0), [0, 7, 30]),
        "empty_wake": (gl, np.zeros((0, 3)), np.array(W.GLIDER_X0), [0, 1, 2]),
        # the perch benchmark's shape (Table I): clean start, merging above 60 particles
        "table1_merging": (dict(gl, n_wake_max=60), np.zeros((0, 3)), np.array(W.GLIDER_X0),
                           [0, 29, 30, 31, 55, 79]),
    }


CASES = _cases()


def _snapshots(ora, params, parts, xg, steps, seed=7):
    cap = len(parts) + 2 * (max(steps) + 2)
    s = ora.State(params, parts, xg, cap)
    rng = np.random.default_rng(seed)
    u = rng.normal(0.0, 3.0, max(steps) + 1)
    snaps = []
    for k in range(max(steps) + 1):
        if k in steps:
            snaps.append((k, snapshot(s), float(u[k])))
        s.step(float(u[k]))
    return snaps, cap


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", sorted(CASES))
def test_step_parity(ora, case, precision):
    torch, V = cuda()
    params, parts, xg, steps = CASES[case]
    snaps, cap = _snapshots(ora, params, parts, xg, steps)
    tol = VEL_TOL if precision == V.FP32 else 1e-11
    for k, snap, u in snaps:
        o = oracle_state(ora, params, snap, cap)
        xg_before, gb_before, hp_before = o.xg.copy(), o.gb_prev.copy(), o.has_prev
        ref = o.step(u)
        g = gpu_state(V, params, snap, cap, precision)
        out = g.step(u, probe=True)
        torch.cuda.synchronize()
        n1 = len(ref["vel"])
        vt = out["vtilde"].cpu().numpy().reshape(-1, 2)
        gs = out["gamma_s"].cpu().numpy()
        fm = out["fm"].cpu().numpy()
        vel = out["vel"].cpu().numpy()[:2 * n1].reshape(-1, 2)
        msg = "%s step %d" % (case, k)
        assert normwise(vt, ref["vtilde"]) <= tol, msg
        assert np.abs(gs - ref["gamma_s"]).max() <= tol * max(1e-3, np.abs(ref["gamma_s"]).max()), msg
        # loads carry the one-step difference quotients of Eq. 13, which divide the surface
        # circulation error by dt
        f_scale = max(1.0, np.abs(ref["fm"]).max())
        assert np.abs(fm - ref["fm"]).max() <= (tol / p_dt(params)) * f_scale, msg
        # the oracle's Eqs. 13-15 applied to the kernel's own surface circulations and plate
        # velocities: both sides form the loads in binary64 from identical inputs, so they agree
        # to rounding (relative to the size of the panel terms, whose difference quotients
        # divide Gamma by dt), and a wrong term, sign or running-sum order in the kernel's
        # pressure, load or moment fails here in either precision
        fm_same = ora.plate_loads(params, xg_before, gs, gb_before, hp_before, vt)
        term = params["rho"] * params["span"] * params["chord"] * (
            np.abs(gs).sum() / p_dt(params) + np.abs(gs).sum() * np.abs(vt).max())
        assert np.abs(fm - fm_same).max() <= 1e-12 * max(1.0, term, np.abs(fm_same).max()), msg
        assert normwise(vel, ref["vel"]) <= tol, msg
        parts_g, xg_g, hist_g = g.read()
        assert len(parts_g) == o.n, msg
        # the advanced positions inherit dt times the velocity tolerance
        vmax = np.linalg.norm(ref["vel"], axis=1).max() if n1 else 0.0
        pos_tol = params["dt"] * tol * vmax + (1e-9 if precision == V.FP32 else 1e-13)
        if len(parts_g):
            assert np.abs(parts_g[:, :2] - o.particles[:, :2]).max() <= pos_tol, msg
            # shed circulations are surface-solve outputs and carry its tolerance
            g_scale = max(1e-3, np.abs(ref["gamma_s"]).max(), np.abs(o.particles[:, 2]).max())
            assert np.abs(parts_g[:, 2] - o.particles[:, 2]).max() <= tol * g_scale, msg
        # glider: dt times the load tolerance divided by the mass (and inertia)
        g_tol = params["dt"] * (tol / params["dt"]) * f_scale / min(params["mass"], params["inertia"])
        assert np.allclose(xg_g, o.xg, rtol=0, atol=g_tol + 1e-12), msg
        g.close()


def p_dt(params):
    return params["dt"]


# Wake sizes at the edges of the binary32 pair phase: its rows of 128 particles (one pair
# evaluation serves both particles across rows), diagonal groups of 64 targets and source
# blocks of 32 (the last one ragged). From 1300 particles on, the row's own pairs are evaluated
# once for both particles too: each size is stepped at n and n + 2, which puts 1298 on both
# sides of that threshold and the others at a last row of 128 (1408), 1 (1409), 32 (1440),
# 33 (1441), 65 (1473) and 97 (1505) particles, i.e. full, empty-tailed and ragged 32-blocks.
ROW_EDGES = [1, 31, 63, 64, 65, 127, 128, 129, 191, 255, 256, 257, 383, 449,
             1298, 1406, 1407, 1438, 1439, 1471, 1503]


@pytest.mark.parametrize("n", ROW_EDGES)
def test_pair_rows_edges(ora, n):
    """One step from the oracle's state at sizes n and n + 2 (after one shedding) against the
    oracle: convection velocities of every particle and the advanced positions."""
    torch, V = cuda()
    params = W.glider_params()
    snaps, cap = _snapshots(ora, params, W.background_field(40 + n, n), np.array(W.GLIDER_X0), [0, 1])
    for k, snap, u in snaps:
        o = oracle_state(ora, params, snap, cap)
        ref = o.step(u)
        g = gpu_state(V, params, snap, cap, V.FP32)
        out = g.step(u, probe=True)
        torch.cuda.synchronize()
        n1 = len(ref["vel"])
        vel = out["vel"].cpu().numpy()[:2 * n1].reshape(-1, 2)
        msg = "n=%d step %d" % (n, k)
        assert normwise(vel, ref["vel"]) <= VEL_TOL, msg
        vmax = np.linalg.norm(ref["vel"], axis=1).max()
        parts_g = g.read()[0]
        assert np.abs(parts_g[:, :2] - o.particles[:, :2]).max() <= params["dt"] * VEL_TOL * vmax + 1e-9, msg
        g.close()


@pytest.mark.parametrize("n", [1298, 1439])
@pytest.mark.parametrize("kernel", ["gaussian", "singular"])
def test_pair_diagonal_other_wake_kernels(ora, kernel, n):
    """The once-per-pair diagonal units (fields of 1300 particles and more) with the Gaussian core
    and the singular kernel of Eq. 4 as the wake kernel: one step at n and n + 2 against the
    oracle. The singular kernel's field is a jittered lattice (no two particles closer than half
    a cell), since binary32 positions leave the 1/r velocity of near-coincident pairs without a
    relative error bound."""
    torch, V = cuda()
    if kernel == "gaussian":
        params = W.glider_params(wake_kernel=W.KERNEL_GAUSSIAN)
        field = W.background_field(70 + n, n)
    else:
        params = W.glider_params(wake_kernel=W.KERNEL_SINGULAR)
        field = W.lattice_field(71 + n, n)
    snaps, cap = _snapshots(ora, params, field, np.array(W.GLIDER_X0), [0, 1])
    for k, snap, u in snaps:
        o = oracle_state(ora, params, snap, cap)
        ref = o.step(u)
        g = gpu_state(V, params, snap, cap, V.FP32)
        out = g.step(u, probe=True)
        torch.cuda.synchronize()
        n1 = len(ref["vel"])
        vel = out["vel"].cpu().numpy()[:2 * n1].reshape(-1, 2)
        msg = "%s n=%d step %d" % (kernel, n, k)
        assert normwise(vel, ref["vel"]) <= VEL_TOL, msg
        g.close()


@pytest.mark.parametrize("n", [3500, 8000])
def test_pair_phase_large_fields(ora, n):
    """Fields above 3000 particles run 512-thread blocks (one per SM) with the once-per-pair
    diagonal units: one step at n and n + 2 from the oracle's state against the oracle, every
    particle's convection velocity and advanced position."""
    torch, V = cuda()
    params = W.glider_params()
    snaps, cap = _snapshots(ora, params, W.background_field(60 + n, n), np.array(W.GLIDER_X0), [0, 1])
    for k, snap, u in snaps:
        o = oracle_state(ora, params, snap, cap)
        ref = o.step(u)
        g = gpu_state(V, params, snap, cap, V.FP32)
        out = g.step(u, probe=True)
        torch.cuda.synchronize()
        n1 = len(ref["vel"])
        vel = out["vel"].cpu().numpy()[:2 * n1].reshape(-1, 2)
        msg = "n=%d step %d" % (n, k)
        assert normwise(vel, ref["vel"]) <= VEL_TOL, msg
        vmax = np.linalg.norm(ref["vel"], axis=1).max()
        parts_g = g.read()[0]
        assert np.abs(parts_g[:, :2] - o.particles[:, :2]).max() <= params["dt"] * VEL_TOL * vmax + 1e-9, msg
        g.close()


def test_step_commits_and_rollout_agree(ora):
    """Ten vpm_step calls advance the resident state exactly as a 10-step rollout does."""
    torch, V = cuda()
    p = W.glider_params()
    field = W.background_field(9, 300)
    g = V.State(p, field, W.GLIDER_X0, 400)
    u = np.linspace(-1, 1, 10).astype(np.float32)
    out = g.rollout_batch(torch.tensor(u[None, :], device="cuda"), want_field=True)
    for k in range(10):
        g.step(float(u[k]))
    parts, xg, _ = g.read()
    n = int(out["count"][0])
    assert n == len(parts) == 320
    assert np.array_equal(out["field"][0, :n].cpu().numpy(), parts)
    assert np.array_equal(out["final_glider"][0].cpu().numpy(), xg)


def test_save_load_resumes_bitwise():
    torch, V = cuda()
    p = W.glider_params()
    g = V.State(p, W.background_field(10, 200), W.GLIDER_X0, 300)
    for k in range(3):
        g.step(0.5)
    blob = g.save()
    for k in range(4):
        g.step(-0.25)
    a = g.read()
    h = V.State(p, np.zeros((0, 3)), np.zeros(7), 300)
    h.load(blob)
    for k in range(4):
        h.step(-0.25)
    b = h.read()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_capacity_rejected_on_host():
    torch, V = cuda()
    g = V.State(W.glider_params(), W.background_field(0, 10), W.GLIDER_X0, 11)
    with pytest.raises(V.VpmError) as e:
        g.step(0.0)
    assert e.value.status == V.VPM_ERR_CAPACITY
    with pytest.raises(V.VpmError) as e:
        g.rollout_batch(torch.zeros((2, 3), device="cuda"))
    assert e.value.status == V.VPM_ERR_CAPACITY


def test_nonfinite_input_rejected():
    torch, V = cuda()
    f = W.background_field(0, 10)
    f[3, 1] = np.nan
    with pytest.raises(V.VpmError) as e:
        V.State(W.glider_params(), f, W.GLIDER_X0, 40)
    assert e.value.status == V.VPM_ERR_NONFINITE
