"""The pins catch single-term mistakes in the oracle.

Each case copies oracle/vpm_oracle.c with one deliberate error in the glider's elevator force and
moment arms (§III-B, Eqs. 19-22) or in the pressure jump and loads (§III-A, Eqs. 13-15), builds it
with the oracle's own compiler flags into a temporary directory, and runs the oracle's pin tests
against it (ORACLE_LIB). Each mutant must fail at least one pin. Host only; the oracle under
oracle/ is not modified.
"""
import os
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "vpm_oracle.c")
PINS = ["tests/test_oracle_glider_mppi.py", "tests/test_oracle_impulse.py", "tests/test_oracle_plate.py"]

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
