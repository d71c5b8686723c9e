"""FP64 CPU oracle of the VPM glider rollouts and MPPI reweighting (ctypes wrapper).

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU-baseline leg
use this package. It never imports or calls the CUDA library, and the CUDA library never
uses it. The arithmetic lives in `vpm_oracle.c` (plain C, binary64, no fast-math); this
file only builds that library with gcc and marshals numpy arrays.

Parameter dictionaries come from `workloads` (the shared seeded-input module).

The environment variable ORACLE_LIB, when set, names another build of `vpm_oracle.c` to load
instead (the mutation tests load copies with one deliberate error each and check that the pins
catch it).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vpm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

SINGULAR, VATISTAS, GAUSSIAN = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile vpm_oracle.c into liboracle.so (gcc, -O2, strict IEEE); with ORACLE_LIB set,
    return that library instead."""
    if os.environ.get("ORACLE_LIB"):
        return os.environ["ORACLE_LIB"]
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
            "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("n_b", C.c_int), ("chord", C.c_double), ("span", C.c_double), ("rho", C.c_double),
        ("wake_kernel", C.c_int), ("r_core", C.c_double), ("shed_offset", C.c_double),
        ("gamma_decay", C.c_double), ("shed_gate", C.c_int), ("alpha_crit", C.c_double),
        ("n_wake_max", C.c_int), ("u_inf_x", C.c_double), ("u_inf_z", C.c_double),
        ("dt", C.c_double), ("fixed_plate", C.c_int),
        ("mass", C.c_double), ("inertia", C.c_double), ("g", C.c_double), ("l", C.c_double),
        ("l_w", C.c_double), ("l_e", C.c_double), ("s_e", C.c_double),
        ("q", C.c_double * 7), ("x_d", C.c_double * 7),
    ]


def make_params(d: dict) -> Params:
    p = Params()
    for k in ("n_b", "wake_kernel", "shed_gate", "n_wake_max", "fixed_plate"):
        setattr(p, k, int(d[k]))
    for k in ("chord", "span", "rho", "r_core", "shed_offset", "gamma_decay", "alpha_crit",
              "dt", "mass", "inertia", "g", "l", "l_w", "l_e", "s_e"):
        setattr(p, k, float(d[k]))
    p.u_inf_x, p.u_inf_z = (float(v) for v in d["u_inf"])
    for i in range(7):
        p.q[i] = float(d["q"][i])
        p.x_d[i] = float(d["x_d"][i])
    return p


_lib = None
_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_DP = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.ora_kernel.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, _DP, _DP]
        L.ora_free_velocity.argtypes = [C.c_int, _D, _D, _D, C.c_int, C.c_double, _D, _D]
        L.ora_velocity_at.argtypes = [C.c_int, _D, _D, _D, C.c_int, C.c_double, C.c_int, _D, _D,
                                      C.c_void_p, _D, _D]
        L.ora_free_euler.argtypes = [C.c_int, _D, _D, _D, C.c_int, C.c_double, C.c_double, C.c_int]
        L.ora_free_heun.argtypes = L.ora_free_euler.argtypes
        L.ora_plate_geometry.argtypes = [C.POINTER(Params), _D, _D]
        L.ora_glider_rhs.argtypes = [C.POINTER(Params), _D, C.c_double, C.c_double, C.c_double,
                                     C.c_double, _D]
        L.ora_plate_loads.argtypes = [C.POINTER(Params), _D, _D, _D, C.c_int, _D, _D]
        L.ora_terminal_cost.argtypes = [C.POINTER(Params), _D]
        L.ora_terminal_cost.restype = C.c_double
        L.ora_step.argtypes = [C.POINTER(Params), C.c_int, C.POINTER(C.c_int), _D, _D, _D, _D, _D,
                               _DP, C.POINTER(C.c_int), C.c_double,
                               C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.POINTER(C.c_int)]
        L.ora_step_dist.argtypes = L.ora_step.argtypes + [C.POINTER(C.c_int)]
        L.ora_rollout.argtypes = [C.POINTER(Params), C.c_int, C.c_int, _D, _D, _D, _D, C.c_void_p,
                                  C.c_double, C.c_int, C.c_int, _D, _D, _DP, C.c_void_p,
                                  C.POINTER(C.c_int), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.ora_mppi_weights.argtypes = [C.c_int, _D, C.c_double, _D]
        L.ora_mppi_update.argtypes = [C.c_int, C.c_int, _D, _D, _D]
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ------------------------------------------------------------------ kernels / free field
def kernel(kind: int, r_core: float, dx: float, dz: float):
    """Velocity (u, w) induced at displacement (dx, dz) by a unit vortex."""
    kx, kz = C.c_double(), C.c_double()
    lib().ora_kernel(kind, r_core, dx, dz, C.byref(kx), C.byref(kz))
    return kx.value, kz.value


def free_velocity(parts, kind: int, r_core: float):
    """Velocity of each particle of a free field (rows x, z, Gamma) from all others."""
    parts = _f64(parts)
    x, z, g = (_f64(parts[:, i]) for i in range(3))
    n = len(x)
    u, w = np.zeros(n), np.zeros(n)
    lib().ora_free_velocity(n, x, z, g, kind, r_core, u, w)
    return np.stack([u, w], axis=1)


def velocity_at(parts, targets, kind: int, r_core: float, skip=None):
    """Velocity at target points (m, 2) from the particles; skip[t] = self index or -1."""
    parts = _f64(parts)
    x, z, g = (_f64(parts[:, i]) for i in range(3))
    t = _f64(targets)
    tx, tz = _f64(t[:, 0]), _f64(t[:, 1])
    m = len(tx)
    u, w = np.zeros(m), np.zeros(m)
    sk = None if skip is None else np.ascontiguousarray(skip, dtype=np.int64)
    lib().ora_velocity_at(len(x), x, z, g, kind, r_core, m, tx, tz, _ptr(sk), u, w)
    return np.stack([u, w], axis=1)


def free_euler(parts, kind, r_core, dt, steps):
    parts = _f64(parts)
    x, z, g = (_f64(parts[:, i]) for i in range(3))
    lib().ora_free_euler(len(x), x, z, g, kind, r_core, dt, steps)
    return np.stack([x, z, g], axis=1)


def free_heun(parts, kind, r_core, dt, steps):
    parts = _f64(parts)
    x, z, g = (_f64(parts[:, i]) for i in range(3))
    lib().ora_free_heun(len(x), x, z, g, kind, r_core, dt, steps)
    return np.stack([x, z, g], axis=1)


# ------------------------------------------------------------------ plate / glider
def plate_geometry(params: dict, xg):
    """Plate points from the glider state; returns a dict of arrays."""
    nb = int(params["n_b"])
    nc = nb + 1
    out = np.zeros(9 + 2 * nc + 2 * nb + 4)
    P = make_params(params)
    lib().ora_plate_geometry(C.byref(P), _f64(xg), out)
    k = 9
    d = dict(xw=out[0:2].copy(), t=out[2:4].copy(), n=out[4:6].copy(), v=out[6:8].copy(),
             omega=out[8])
    d["c"] = np.stack([out[k:k + nc], out[k + nc:k + 2 * nc]], axis=1); k += 2 * nc
    d["b"] = np.stack([out[k:k + nb], out[k + nb:k + 2 * nb]], axis=1); k += 2 * nb
    d["lev"] = out[k:k + 2].copy(); d["tev"] = out[k + 2:k + 4].copy()
    return d


def plate_loads(params: dict, xg, gamma_s, gb_prev, has_prev: int, vtilde):
    """Wing load and moment (F_w,x, F_w,z, M_w) of Eqs. 13-15 from given surface circulations
    (N_b bound, Gamma_LEV, Gamma_TEV), previous bound circulations and plate-point relative
    velocities (N_b + 1 collocation points, then N_b bound points, as (u, w) rows)."""
    fm = np.zeros(3)
    P = make_params(params)
    lib().ora_plate_loads(C.byref(P), _f64(xg), _f64(gamma_s), _f64(gb_prev), int(has_prev),
                          _f64(np.asarray(vtilde).reshape(-1)), fm)
    return fm


def glider_rhs(params: dict, xg, fw, mw, u):
    f = np.zeros(7)
    P = make_params(params)
    lib().ora_glider_rhs(C.byref(P), _f64(xg), float(fw[0]), float(fw[1]), float(mw), float(u), f)
    return f


def terminal_cost(params: dict, xg) -> float:
    P = make_params(params)
    return lib().ora_terminal_cost(C.byref(P), _f64(xg))


class State:
    """Coupled glider + wake state advanced by `step` (one call of the C oracle per step)."""

    def __init__(self, params: dict, parts, xg, capacity: int, gb_prev=None, glev_prev=0.0,
                 has_prev=0, n_dist=0):
        self.params = dict(params)
        self._P = make_params(params)
        parts = _f64(parts).reshape(-1, 3)
        self.capacity = int(capacity)
        self.n = len(parts)
        self.x = np.zeros(self.capacity); self.z = np.zeros(self.capacity)
        self.g = np.zeros(self.capacity)
        self.x[:self.n], self.z[:self.n], self.g[:self.n] = parts[:, 0], parts[:, 1], parts[:, 2]
        self.xg = _f64(xg).copy()
        nb = int(params["n_b"])
        self.gb_prev = np.zeros(nb) if gb_prev is None else _f64(gb_prev).copy()
        self.glev_prev = float(glev_prev)
        self.has_prev = int(has_prev)
        self.n_dist = int(n_dist)       # 2: the first two particles are the disturbance pair

    @property
    def particles(self):
        return np.stack([self.x[:self.n], self.z[:self.n], self.g[:self.n]], axis=1)

    def copy(self):
        s = State(self.params, self.particles, self.xg, self.capacity, self.gb_prev,
                  self.glev_prev, self.has_prev, self.n_dist)
        return s

    def inject_pair(self, x1, z1, g1, x2, z2, g2):
        """Puts a disturbance pair (§V) in front of the wake: particles 0 and 1, left out of
        merging and removed once their segment crosses the offset chord line."""
        if self.n_dist:
            raise ValueError("a disturbance pair is already present")
        if self.n + 2 > self.capacity:
            raise ValueError("capacity exceeded")
        for arr, a, b in ((self.x, x1, x2), (self.z, z1, z2), (self.g, g1, g2)):
            arr[2:self.n + 2] = arr[:self.n].copy()
            arr[0], arr[1] = a, b
        self.n += 2
        self.n_dist = 2

    def step(self, u: float = 0.0):
        """One step; returns dict(gamma_s, fm, vel, vtilde, alpha)."""
        nb = int(self.params["n_b"])
        nc = nb + 1
        gs = np.zeros(nb + 2); fm = np.zeros(3)
        vel = np.zeros(2 * (self.n + 2)); vt = np.zeros(2 * (nc + nb)); al = np.zeros(1)
        n = C.c_int(self.n); gl = C.c_double(self.glev_prev); hp = C.c_int(self.has_prev)
        shed = C.c_int(0)
        nd = C.c_int(self.n_dist)
        n_before = self.n
        rc = lib().ora_step_dist(C.byref(self._P), self.capacity, C.byref(n), self.x, self.z, self.g,
                                 self.xg, self.gb_prev, C.byref(gl), C.byref(hp), float(u),
                                 _ptr(gs), _ptr(fm), _ptr(vel), _ptr(vt), _ptr(al), C.byref(shed),
                                 C.byref(nd))
        if rc != 0:
            raise RuntimeError("oracle step failed with status %d" % rc)
        self.n, self.glev_prev, self.has_prev = n.value, gl.value, hp.value
        self.n_dist = nd.value
        m = n_before + shed.value
        return dict(gamma_s=gs, fm=fm, vel=vel[:2 * m].reshape(-1, 2),
                    vtilde=vt.reshape(-1, 2), alpha=al[0], shed=shed.value)


def rollout(params: dict, parts, xg0, controls, capacity=None, gb_prev=None, glev_prev=0.0,
            has_prev=0, want_traj=False, want_field=False, n_dist=0):
    """One rollout of len(controls) steps; returns dict(xg, cost, traj?, field?)."""
    parts = _f64(parts).reshape(-1, 3)
    H = len(controls)
    cap = capacity if capacity is not None else len(parts) + 2 * H
    x, z, g = (_f64(parts[:, i]) for i in range(3))
    xg = np.zeros(7); cost = C.c_double()
    traj = np.zeros((H, 7)) if want_traj else None
    fx = np.zeros(cap) if want_field else None
    fz = np.zeros(cap) if want_field else None
    fg = np.zeros(cap) if want_field else None
    nout = C.c_int()
    gbp = None if gb_prev is None else _f64(gb_prev)
    P = make_params(params)
    rc = lib().ora_rollout(C.byref(P), cap, len(x), x, z, g, _f64(xg0), _ptr(gbp),
                           float(glev_prev), int(has_prev), H, _f64(controls), xg,
                           C.byref(cost), _ptr(traj), C.byref(nout), _ptr(fx), _ptr(fz), _ptr(fg),
                           int(n_dist))
    if rc != 0:
        raise RuntimeError("oracle rollout failed with status %d" % rc)
    out = dict(xg=xg, cost=cost.value)
    if want_traj:
        out["traj"] = traj
    if want_field:
        n = nout.value
        out["field"] = np.stack([fx[:n], fz[:n], fg[:n]], axis=1)
    return out


# ------------------------------------------------------------------ MPPI
def mppi_weights(J, lam: float):
    J = _f64(J)
    w = np.zeros(len(J))
    lib().ora_mppi_weights(len(J), J, float(lam), w)
    return w


def mppi_update(w, xi):
    w = _f64(w)
    xi = _f64(xi)
    K, H = xi.shape
    mu = np.zeros(H)
    lib().ora_mppi_update(K, H, w, xi, mu)
    return mu
