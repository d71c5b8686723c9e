"""The pins catch single-term mistakes in the oracle.

Each case copies oracle/vpm_oracle.c with one deliberate error: in the kernels (Eqs. 4-5 and the
Gaussian core), the free-field integrators, the plate geometry and relative velocity (Eq. 12), the
surface system and Kelvin's row (Eqs. 6-11), the pressure jump and loads (Eqs. 13-15), convection,
decay and merging (Eqs. 16-17), the glider's elevator force, moment arms and equations of motion
(Eqs. 18-22), the terminal cost (Eq. 24), MPPI (Eq. 25), the separation gate or the linear solve. It
builds the copy with the oracle's own compiler flags into a temporary directory and runs the
oracle's pin tests against it (ORACLE_LIB). The Python parts of the oracle (the tracking policy of
§IV-B in oracle/policy.py, the NMPC loop of §IV-C in oracle/nmpc.py) get the same treatment: each
case edits a copy of the oracle, the tests and the input generators in a temporary directory and
runs the pins there. Each mutant must fail at least one pin. Host only; the oracle under oracle/ is
not modified.
"""
import glob
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "vpm_oracle.c")
PINS = sorted(os.path.relpath(f, ROOT) for f in glob.glob(os.path.join(ROOT, "tests", "test_oracle_*.py"))
              if not f.endswith("test_oracle_mutations.py")) + ["tests/test_golden.py"]

# (name, exact text in vpm_oracle.c, replacement)
MUTATIONS = [
    ("elevator: the 1/2 of the dynamic pressure dropped",
     "double q = 0.5 * p->rho * (xed * xed + zed * zed) * p->s_e * cn;",
     "double q = p->rho * (xed * xed + zed * zed) * p->s_e * cn;"),
    ("elevator: C_n = sin(alpha_e)", "double cn = 2.0 * sin(alpha_e);", "double cn = sin(alpha_e);"),
    ("elevator: area doubled", "* p->s_e * cn;", "* 2.0 * p->s_e * cn;"),
    ("elevator: incidence sign", "double alpha_e = th + ph - atan2(zed, xed);",
     "double alpha_e = atan2(zed, xed) - th - ph;"),
    ("pitch: elevator arm without the elevator's own length",
     "double aex = -p->l * ct - p->l_e * cp, aez = -p->l * st - p->l_e * sp;",
     "double aex = -p->l * ct, aez = -p->l * st;"),
    ("pitch: wing arm reversed", "double awx = -p->l_w * ct, awz = -p->l_w * st;",
     "double awx = p->l_w * ct, awz = p->l_w * st;"),
    ("Eq. 13: dGamma_LEV/dt dropped", "double dlev = has_prev ? gs[nb] / dt : 0.0;", "double dlev = 0.0;"),
    ("Eq. 13: dGamma_LEV/dt negated", "double dlev = has_prev ? gs[nb] / dt : 0.0;",
     "double dlev = has_prev ? -gs[nb] / dt : 0.0;"),
    ("Eq. 13: dGamma_LEV/dt halved", "double dlev = has_prev ? gs[nb] / dt : 0.0;",
     "double dlev = has_prev ? 0.5 * gs[nb] / dt : 0.0;"),
    ("Eq. 13: bound running sums' derivative dropped", "double dsum = has_prev ? (cum - cum_prev) / dt : 0.0;",
     "double dsum = 0.0;"),
    ("Eq. 13: bound running sums' derivative negated", "double dsum = has_prev ? (cum - cum_prev) / dt : 0.0;",
     "double dsum = has_prev ? (cum_prev - cum) / dt : 0.0;"),
    ("Eq. 13: tangential term's sign", "double dp = p->rho * (tang + dsum + dlev);",
     "double dp = p->rho * (-tang + dsum + dlev);"),
    ("Eq. 15: moment's sign", "mw += ax * fz - az * fx;", "mw -= ax * fz - az * fx;"),
    # the rest of the oracle
 ("singular kernel sign", "double s = -1.0 / (2.0 * ORA_PI * r2);", "double s = 1.0 / (2.0 * ORA_PI * r2);"),
 ("singular kernel components swapped", "    *kx = s * jx;\n    *kz = s * jz;", "    *kx = s * jz;\n    *kz = s * jx;"),
 ("singular kernel 1/(pi r^2)", "double s = -1.0 / (2.0 * ORA_PI * r2);", "double s = -1.0 / (ORA_PI * r2);"),
 ("Vatistas exponent", "return q / sqrt(1.0 + q * q);", "return q / sqrt(1.0 + q);"),
 ("Gaussian core in r", "return 1.0 - exp(-(r * r) / (rc * rc));", "return 1.0 - exp(-r / rc);"),
 ("Heun second stage only", "            x[i] += 0.5 * dt * (u1[i] + u2[i]);", "            x[i] += dt * u2[i];"),
 ("Euler z sign", "for (int i = 0; i < n; ++i) { x[i] += dt * u[i]; z[i] += dt * w[i]; }", "for (int i = 0; i < n; ++i) { x[i] += dt * u[i]; z[i] -= dt * w[i]; }"),
 ("normal reversed", "G->nx = -s;  G->nz = c;", "G->nx = s;  G->nz = -c;"),
 ("bound vortices at collocation points", "double sj = -0.5 * p->chord + (j + 0.5) * G->lb;", "double sj = -0.5 * p->chord + j * G->lb;"),
 ("LEV on the wrong side", "G->lev_x = G->cx[0] - ds * G->tx;\n    G->lev_z = G->cz[0] - ds * G->tz;", "G->lev_x = G->cx[0] + ds * G->tx;\n    G->lev_z = G->cz[0] + ds * G->tz;"),
 ("plate velocity rotation sign", "G->vx = xg[4] + p->l_w * xg[6] * s;\n        G->vz = xg[5] - p->l_w * xg[6] * c;", "G->vx = xg[4] - p->l_w * xg[6] * s;\n        G->vz = xg[5] + p->l_w * xg[6] * c;"),
 ("Eq. 12 rotation term sign", "*u = wu + p->u_inf_x - G->vx - G->omega * ex;\n    *w = ww + p->u_inf_z - G->vz - G->omega * ez;", "*u = wu + p->u_inf_x - G->vx + G->omega * ex;\n    *w = ww + p->u_inf_z - G->vz + G->omega * ez;"),
 ("Eq. 12 free stream dropped", "*u = wu + p->u_inf_x - G->vx - G->omega * ex;\n    *w = ww + p->u_inf_z - G->vz - G->omega * ez;", "*u = wu - G->vx - G->omega * ex;\n    *w = ww - G->vz - G->omega * ez;"),
 ("Kelvin row sign", "    b[r] = -gw;", "    b[r] = gw;"),
 ("no-through-flow right-hand side sign", "b[r] = -(vcx[i] * G.nx + vcz[i] * G.nz);", "b[r] = (vcx[i] * G.nx + vcz[i] * G.nz);"),
 ("shed vortices' columns with the singular kernel", "kernel_eval(p->wake_kernel, p->r_core, G.cx[i] - G.lev_x, G.cz[i] - G.lev_z, &kx, &kz);", "kernel_eval(ORA_SINGULAR, 0.0, G.cx[i] - G.lev_x, G.cz[i] - G.lev_z, &kx, &kz);"),
 ("bound vortices left out of the convection", "uu[i] = su + bu + p->u_inf_x;\n        ww[i] = sw + bw + p->u_inf_z;", "uu[i] = su + p->u_inf_x;\n        ww[i] = sw + p->u_inf_z;"),
 ("decay grows", "double decay = exp(-p->gamma_decay * dt);", "double decay = exp(p->gamma_decay * dt);"),
 ("merge keeps the newer position", "x[d] = 0.5 * (x[d] + x[d + 1]);\n            z[d] = 0.5 * (z[d] + z[d + 1]);", "x[d] = x[d + 1];\n            z[d] = z[d + 1];"),
 ("merge averages the circulation", "g[d] = g[d] + g[d + 1];", "g[d] = 0.5 * (g[d] + g[d + 1]);"),
 ("gravity sign", "f[5] = (fwz + fez) / p->mass - p->g;", "f[5] = (fwz + fez) / p->mass + p->g;"),
 ("pitch divided by the mass", "f[6] = torque / p->inertia;", "f[6] = torque / p->mass;"),
 ("MPPI exponent sign", "? exp(-(J[i] - jmin) / lambda) : 0.0;", "? exp((J[i] - jmin) / lambda) : 0.0;"),
 ("MPPI: a diverged rollout keeps a weight", "? exp(-(J[i] - jmin) / lambda) : 0.0;", "? exp(-(J[i] - jmin) / lambda) : 1e-300;"),
 ("MPPI: J_min taken over every cost", "if (isfinite(J[i])) { finite = 1; if (J[i] < jmin) jmin = J[i]; }",
  "{ finite |= isfinite(J[i]) != 0; if (J[i] < jmin) jmin = J[i]; }"),
 ("MPPI not normalised", "double eta = 1.0 / s;", "double eta = 1.0;"),
 ("cost weights squared", "J += d * p->q[k] * d;", "J += d * p->q[k] * p->q[k] * d;"),
 ("gate mode 2 stops the TEV too", "int shed_tev = (p->shed_gate != 1) || open;", "int shed_tev = (p->shed_gate == 0) || open;"),
 ("LU pivot not swapped in b", "double t = b[k]; b[k] = b[piv]; b[piv] = t;", "double t = b[k]; (void)t;"),
 ("MPPI update transposed", "s += w[i] * xi[(size_t)i * H + k];", "s += w[i] * xi[(size_t)k * K + i];"),
]

# (name, file under oracle/, [(exact text, replacement), ...])
PY_MUTATIONS = [
    ("policy law: feedback sign", "policy.py",
     [("return float(ubar[k]) - float(", "return float(ubar[k]) + float(")]),
    ("policy rollout: feedback sign", "policy.py",
     [("u = float(ubar[j]) - float(np.asarray(gains[j])", "u = float(ubar[j]) + float(np.asarray(gains[j])")]),
    ("policy rollout: policy rows one step ahead", "policy.py",
     [("        j = offset + k\n", "        j = min(offset + k + 1, len(gains) - 1)\n")]),
    ("policy rollout: nominal states one step behind", "policy.py",
     [("(s.xg - np.asarray(xbar[j])))", "(s.xg - np.asarray(xbar[max(j - 1, 0)])))")]),
    ("Euler discretisation: B not scaled by dt", "policy.py",
     [("return np.eye(STATE) + dt * A, dt * B", "return np.eye(STATE) + dt * A, B")]),
    ("TVLQR: control weight dropped", "policy.py", [("denom = rc + B @ Sn @ B", "denom = B @ Sn @ B")]),
    ("TVLQR: running cost dropped", "policy.py",
     [("np.outer(A.T @ Sn @ B, B @ Sn @ A) / denom + Qc", "np.outer(A.T @ Sn @ B, B @ Sn @ A) / denom")]),
    ("least squares: derivative of the nominal one step late", "policy.py",
     [("xbar_dot = (xbar[k + 1] - xbar[k]) / dt", "xbar_dot = (xbar[min(k + 2, len(xbar) - 1)] - xbar[k + 1]) / dt")]),
    ("structure: kinematic identity on the positions", "policy.py",
     [("A[0, 4] = A[1, 5] = A[2, 6] = 1.0", "A[0, 0] = A[1, 1] = A[2, 2] = 1.0")]),
    ("NMPC: policy rows one step ahead", "nmpc.py",
     [("        j = t - self.t0\n", "        j = min(t - self.t0 + 1, len(self.gains) - 1)\n")]),
    ("NMPC: a plan takes effect the step after it is made", "nmpc.py",
     [("        if pending is not None and t == pending.t0:\n", "        if pending is not None:\n")]),
    ("NMPC: a due plan takes effect after the replan of its step", "nmpc.py",
     [("        if pending is not None and t == pending.t0:\n            pol, pending = pending, None\n"
       "        if t > 0", "        if t > 0"),
      ("        u = pol.control(t, x_obs)\n", "        if pending is not None and t == pending.t0:\n"
       "            pol, pending = pending, None\n        u = pol.control(t, x_obs)\n")]),
    ("NMPC: a plan made with no latency waits a step", "nmpc.py",
     [("            if L == 0:\n                pol, pending = pending, None\n", "")]),
    ("NMPC: projection one step short", "nmpc.py", [("            for k in range(L):\n", "            for k in range(max(L - 1, 0)):\n")]),
    ("NMPC: projection under the nominal controls alone", "nmpc.py",
     [("snap.step(pol.control(t + k, snap.xg))", "snap.step(float(pol.ubar[t + k]))")]),
    ("NMPC: projection from the tracking instance's own glider state", "nmpc.py",
     [("            snap.xg[:] = x_obs\n", "")]),
    ("NMPC: tracking instance not reset to the observed state", "nmpc.py",
     [("        tracking.xg[:] = x_obs\n", "")]),
    ("NMPC: warm start from the initial controls", "nmpc.py",
     [("plan(cfg, params, snap, mu, t + L, noise[used])", "plan(cfg, params, snap, mu0, t + L, noise[used])")]),
    ("NMPC: a replan reuses the previous plan's draws", "nmpc.py",
     [("plan(cfg, params, snap, mu, t + L, noise[used])", "plan(cfg, params, snap, mu, t + L, noise[used - 1])")]),
    ("NMPC: perturbations indexed by absolute step", "nmpc.py", [("eps[it][:, :Hr]", "eps[it][:, t0:]")]),
    ("NMPC: nominal states without the snapshot's state", "nmpc.py",
     [('xbar = np.vstack([snap.xg, nom["traj"]])', 'xbar = np.vstack([nom["traj"][:1], nom["traj"]])')]),
    ("NMPC: replan at t = 0", "nmpc.py", [("if t > 0 and t % Pn == 0", "if t % Pn == 0")]),
    ("NMPC: replan while t + L <= N", "nmpc.py", [("t + L < N and used", "t + L <= N - 1 + (L > 0) and used")]),
]


def _mutant(tmp, k, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, old
    path = os.path.join(tmp, "mutant%d.c" % k)
    open(path, "w").write(src.replace(old, new))
    lib = os.path.join(tmp, "libmutant%d.so" % k)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                           "-ffp-contract=off", "-o", lib, path, "-lm"])
    return lib


def _py_mutant(tmp, k, rel, edits):
    """A copy of oracle/, tests/, workloads/ and pytest.ini with the edits made to oracle/rel."""
    dst = os.path.join(tmp, "py%d" % k)
    skip = shutil.ignore_patterns("__pycache__", "*.so", "*.tmp*")
    for d in ("oracle", "tests", "workloads"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(dst, d), ignore=skip)
    shutil.copy(os.path.join(ROOT, "pytest.ini"), dst)
    path = os.path.join(dst, "oracle", rel)
    src = open(path).read()
    for old, new in edits:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    open(path, "w").write(src)
    return dst


def _pins_against(lib, cwd=ROOT):
    env = dict(os.environ, ORACLE_LIB=lib)
    env.pop("PYTHONPATH", None)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"] + PINS, cwd=cwd, env=env, capture_output=True, text=True,
                       timeout=600)
    return r.returncode, r.stdout[-400:]


def test_every_single_term_mutation_fails_a_pin():
    with tempfile.TemporaryDirectory() as tmp:
        libs = [_mutant(tmp, k, old, new) for k, (_, old, new) in enumerate(MUTATIONS)]
        with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
            results = list(ex.map(_pins_against, libs))
    survivors = [(name, out) for (name, _, _), (rc, out) in zip(MUTATIONS, results) if rc == 0]
    assert not survivors, survivors
    # every run failed a test, none died on something else
    assert all(rc == 1 for rc, _ in results), [out for rc, out in results if rc != 1]


def test_every_python_oracle_mutation_fails_a_pin(ora):
    lib = ora.build()
    with tempfile.TemporaryDirectory() as tmp:
        dirs = [_py_mutant(tmp, k, rel, edits) for k, (_, rel, edits) in enumerate(PY_MUTATIONS)]
        # the unmodified copy passes, so the failures below come from the edits
        clean = _py_mutant(tmp, len(PY_MUTATIONS), "nmpc.py", [])
        with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
            results = list(ex.map(lambda d: _pins_against(lib, d), dirs + [clean]))
    assert results[-1][0] == 0, results[-1][1]
    results = results[:-1]
    survivors = [(name, out) for (name, _, _), (rc, out) in zip(PY_MUTATIONS, results) if rc == 0]
    assert not survivors, survivors
    assert all(rc == 1 for rc, _ in results), [out for rc, out in results if rc != 1]
