"""Small numpy restatements used to pin the oracle from outside.

They are written from the textbook forms, not from the oracle's code: the point-vortex
velocity as the cross product of Eq. 2, -(1/2pi) (r - r_v) x (Gamma e_y) / |r - r_v|^2, in
3-D with numpy's cross product (the plane is (x, z); the paper's out-of-plane unit vector
e_z of §III-A is the third axis here), and the core factors as functions of r.
"""
import math

import numpy as np

# In the (x, z) plane with z up, the out-of-plane axis that makes circulation positive
# counter-clockwise is -y in a right-handed (x, y, z) frame: e_x x e_z = -e_y.
_OUT = np.array([0.0, -1.0, 0.0])


def core_factor(kind: int, r, rc):
    r = np.asarray(r, dtype=np.float64)
    if kind == 0:
        return np.ones_like(r)
    if kind == 1:
        return r ** 2 / np.sqrt(rc ** 4 + r ** 4)
    return -np.expm1(-(r / rc) ** 2)


def biot_savart(src, targets, kind: int, rc: float, skip_self: bool = False):
    """Velocity at targets (m, 2) from sources (n, 3) via 3-D cross products."""
    src = np.asarray(src, dtype=np.float64)
    tgt = np.asarray(targets, dtype=np.float64)
    d = tgt[:, None, :] - src[None, :, :2]                       # (m, n, 2) in (x, z)
    d3 = np.stack([d[..., 0], np.zeros_like(d[..., 0]), d[..., 1]], axis=-1)
    zeta = src[:, 2][None, :, None] * _OUT[None, None, :]        # Gamma along the out axis
    cr = np.cross(d3, np.broadcast_to(zeta, d3.shape))
    r2 = (d ** 2).sum(-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        v3 = -cr / (2 * math.pi * r2[..., None])
        v3 = v3 * core_factor(kind, np.sqrt(r2), rc)[..., None]
    v3[r2 == 0] = 0.0
    if skip_self:
        m = min(len(tgt), len(src))
        v3[np.arange(m), np.arange(m)] = 0.0
    v = v3.sum(1)
    return np.stack([v[:, 0], v[:, 2]], axis=1)


def wagner_jones(s):
    """R. T. Jones' two-exponential approximation of Wagner's indicial lift function,
    s = distance travelled in semichords."""
    return 1.0 - 0.165 * np.exp(-0.0455 * s) - 0.335 * np.exp(-0.3 * s)


def vortex_impulse(points, gammas):
    """Hydrodynamic impulse per unit density and span of a system of point vortices in the
    plane: P = sum_k Gamma_k r_k x e_out, with e_out the out-of-plane axis about which
    circulation is positive (counter-clockwise in the (x, z) plane, z up). In (x, z)
    components, r x e_out = (z, -x). The fluid's momentum changes only by the force the
    body exerts on it, so the force of the fluid on the body is -rho s dP/dt."""
    pts = np.asarray(points, dtype=np.float64).reshape(-1, 2)
    g = np.asarray(gammas, dtype=np.float64).reshape(-1)
    return np.array([(g * pts[:, 1]).sum(), -(g * pts[:, 0]).sum()])


def elevator_point(xg, l, l_e):
    """Elevator point of the planar glider: the tail hinge lies l behind the centre of gravity
    along the body axis (cos theta, sin theta), the elevator point l_e behind the hinge along
    the elevator chord (cos(theta + phi), sin(theta + phi))."""
    x, z, th, ph = xg[0], xg[1], xg[2], xg[3]
    return np.array([x - l * math.cos(th) - l_e * math.cos(th + ph),
                     z - l * math.sin(th) - l_e * math.sin(th + ph)])


def wing_point(xg, l_w):
    """Wing centre: l_w behind the centre of gravity along the body axis."""
    x, z, th = xg[0], xg[1], xg[2]
    return np.array([x - l_w * math.cos(th), z - l_w * math.sin(th)])


def point_velocity(point_of, xg, u, h=1e-6):
    """Velocity of a body point by a central difference along the state's own motion
    (constant rates xdot, zdot, thetadot and elevator rate u over +-h)."""
    xg = np.asarray(xg, dtype=np.float64)
    rate = np.array([xg[4], xg[5], xg[6], u, 0.0, 0.0, 0.0])
    return (point_of(xg + h * rate) - point_of(xg - h * rate)) / (2 * h)


def cross2(a, b):
    """Planar cross product a x b = a_x b_z - a_z b_x (counter-clockwise positive)."""
    return a[0] * b[1] - a[1] * b[0]
