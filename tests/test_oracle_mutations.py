"""The pins catch single-term mistakes in the oracle.

Each case copies oracle/vpm_oracle.c with one deliberate error: in the kernels (Eqs. 4-5 and the
Gaussian core), the free-field integrators, the plate geometry and relative velocity (Eq. 12), the
surface system and Kelvin's row (Eqs. 6-11), the pressure jump and loads (Eqs. 13-15), convection,
decay and merging (Eqs. 16-17), the glider's elevator force, moment arms and equations of motion
(Eqs. 18-22), the terminal cost (Eq. 24), MPPI (Eq. 25), the separation gate or the linear solve. It
builds the copy with the oracle's own compiler flags into a temporary directory and runs the
oracle's pin tests against it (ORACLE_LIB). Each mutant must fail at least one pin. Host only; the
oracle under oracle/ is not modified.
"""
import glob
import os
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
 ("MPPI exponent sign", "w[i] = exp(-(J[i] - jmin) / lambda);", "w[i] = exp((J[i] - jmin) / lambda);"),
 ("MPPI not normalised", "double eta = 1.0 / s;", "double eta = 1.0;"),
 ("cost weights squared", "J += d * p->q[k] * d;", "J += d * p->q[k] * p->q[k] * d;"),
 ("gate mode 2 stops the TEV too", "int shed_tev = (p->shed_gate != 1) || open;", "int shed_tev = (p->shed_gate == 0) || open;"),
 ("LU pivot not swapped in b", "double t = b[k]; b[k] = b[piv]; b[piv] = t;", "double t = b[k]; (void)t;"),
 ("MPPI update transposed", "s += w[i] * xi[(size_t)i * H + k];", "s += w[i] * xi[(size_t)k * K + i];"),
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


def _pins_against(lib):
    env = dict(os.environ, ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"] + PINS, cwd=ROOT, env=env, capture_output=True, text=True,
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
