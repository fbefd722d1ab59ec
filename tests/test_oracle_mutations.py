"""The pins catch plausible mistakes in the oracle (CPU, no GPU).

Each case plants one mistake in a copy of oracle/dgsrhd_oracle.c (a wrong Runge-Kutta weight,
a flipped dissipation sign, a transposed or swapped basis table, face traces from the wrong
face, a wrong wavespeed, enthalpy, pressure or quadratic factor, a looser Newton stop, the HLLC
star state on the wrong side or with a wrong sign, the operator's other root or a missing
margin, its face-point variant without the face points or with the end nodes for them, the
limiter's bound scaling, the minmod limiter's threshold, sign test and differences),
or in a copy of oracle/exact_riemann_general.py (the
rarefaction ODE, the isentrope, the shock speed, the transverse invariant behind a shock), builds
the copy in a temporary directory, and runs the fast pin files against it in
a child process whose oracle module loads that copy.  Every planted mistake must make at least
one pin fail, and an unmodified copy must pass them all, so a failure here means a pin has
stopped testing what it claims to.  The planted copies never leave the temporary directory.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SOURCE = os.path.join(ROOT, "oracle", "dgsrhd_oracle.c")

# (what is wrong, exact text in the source, the mistaken text)
MUTATIONS = [
    ("SSPRK3 final-stage weight", "{0.0, 0.75, 1.0 / 3.0}", "{0.0, 0.75, 0.3}"),
    ("LLF dissipation sign", "- 0.5 * a * (UR[v] - UL[v])", "+ 0.5 * a * (UR[v] - UL[v])"),
    ("HLL dissipation sign", "sL * sR * (UR[v] - UL[v])", "sL * sR * (UL[v] - UR[v])"),
    ("lift with phi(+1) at the low face", "+= scale * (m.em[a] / m.w[a]) * Fs[v]",
     "+= scale * (m.ep[a] / m.w[a]) * Fs[v]"),
    ("volume table transposed", "w[a] * lagrange_deriv(N, x, i, x[a]) / w[i]",
     "w[i] * lagrange_deriv(N, x, a, x[i]) / w[a]"),
    ("wavespeed sigma with one Lorentz factor", "cs2 / (gam * gam * (1.0 - cs2))",
     "cs2 / (gam * (1.0 - cs2))"),
    ("operator takes the other root", "double den = -b + sqrt(b * b - 4.0 * a * c0);",
     "double den = -b - sqrt(b * b - 4.0 * a * c0);"),
    ("operator without its margin", "s *= (1.0 - 1e-12);", "s *= 1.0;"),
    ("Taub-Matthews enthalpy constant",
     "1.5 * th * th / (sqrt(th * th + 4.0 / 9.0) + 2.0 / 3.0)",
     "1.5 * th * th / (sqrt(th * th + 4.0 / 9.0) + 1.0 / 3.0)"),
    ("ideal enthalpy factor", "c->gamma_ad / (c->gamma_ad - 1.0) * th",
     "1.0 / (c->gamma_ad - 1.0) * th"),
    ("ideal pressure from con2prim", "P = (c->gamma_ad - 1.0) * e_minus_rho;",
     "P = c->gamma_ad * e_minus_rho;"),
    ("Taub-Matthews pressure from con2prim", "P = e_minus_rho * (Ev + rho) / (3.0 * Ev);",
     "P = e_minus_rho * (Ev + rho) / (2.0 * Ev);"),
    ("the quartic's other quadratic factor", "double C = 0.5 * (x - sqrt(x * x - 4.0 * a0));",
     "double C = 0.5 * (x + sqrt(x * x - 4.0 * a0));"),
    ("limiter bound scaling h^(3/2)", "pow(h, 1.5)", "pow(h, 2.0)"),
    ("HLLC star state on the wrong side of the contact", "const int left = xs >= 0.0;",
     "const int left = xs < 0.0;"),
    ("HLLC tau* pressure work sign", "Us[4] = (U[4] * (lam - v) + ps * xs - p * v) / den;",
     "Us[4] = (U[4] * (lam - v) + ps * xs + p * v) / den;"),
    ("looser Newton stop", "fabs(dw) <= fmax(1e-14, rtol) * w", "fabs(dw) <= fmax(1e-6, rtol) * w"),
    ("face traces from the opposite face", "const double *coef = side ? m->ep : m->em;",
     "const double *coef = side ? m->em : m->ep;"),
    ("face-point operator leaves the face points out of the minimum",
     "    double si = point_factor(Uf, Ub);\n", "    double si = 1.0;\n"),
    ("face-point operator takes the end node for the face value",
     "out[v] += coef[a] * U[v * tot + e * m->Nn + node];",
     "out[v] += (a == (side ? m->N - 1 : 0)) * U[v * tot + e * m->Nn + node];"),
    ("minmod TVB threshold scaled by h", "const double thr = c->limiter_alpha * h * h;",
     "const double thr = c->limiter_alpha * h;"),
    ("minmod ignores the signs of the neighbour differences",
     "if ((D[k] > 0.0) != (x > 0.0) || D[k] == 0.0) return 0.0;", "if (D[k] == 0.0) return 0.0;"),
    ("minmod backward difference with the wrong sign", "D[nD++] = side ? un - ub : ub - un;",
     "D[nD++] = un - ub;"),
    ("minmod low-face deviation with the wrong sign",
     "const double dev[2] = {fm[1] / face_wsum - ub, ub - fm[0] / face_wsum};",
     "const double dev[2] = {fm[1] / face_wsum - ub, fm[0] / face_wsum - ub};"),
]

# the same for the exact Riemann solution with transverse velocity (a Python module)
EXACT_SOURCE = os.path.join(ROOT, "oracle", "exact_riemann_general.py")
EXACT_MUTATIONS = [
    ("rarefaction ODE without c_s^2 on v_t^2", "math.sqrt(1.0 - vx * vx - c2 * vt * vt)",
     "math.sqrt(1.0 - vx * vx - vt * vt)"),
    ("isentrope without h", "return [p / (rho * h * c2),", "return [p / (rho * c2),"),
    ("shock speed sign under the root", "math.sqrt(j2 + m2 * (1.0 - vx_a * vx_a))",
     "math.sqrt(j2 + m2 * (1.0 + vx_a * vx_a))"),
    ("transverse invariant behind a shock without h", "A = h_a * lor_a * vt_a",
     "A = lor_a * vt_a"),
]
EXACT_PINS = ["tests/test_exact_riemann_general.py"]

PINS = [
    "tests/test_oracle_basis.py", "tests/test_oracle_eos.py", "tests/test_oracle_flux.py",
    "tests/test_oracle_enforce.py", "tests/test_oracle_enforce_faces.py", "tests/test_oracle_rhs.py",
    "tests/test_oracle_con2prim.py",
    "tests/test_oracle_step.py", "tests/test_oracle_limiter.py",
] + [f"tests/test_oracle_minmod.py::{t}" for t in (
    "test_linear_data_untouched", "test_local_extremum_is_flattened_and_means_kept",
    "test_limited_elements_scale_toward_the_mean_within_the_minmod_bound",
    "test_tvb_threshold_keeps_small_deviations", "test_riemann_problem_converges_with_minmod")]

# The child imports the oracle package, points its source and build paths at the copy before
# anything loads the shared object, and runs the pins; the pin modules import the same package.
CHILD = """
import os, sys
sys.path.insert(0, {root!r})
import oracle
oracle._SRC = sys.argv[1]
oracle._BUILD = sys.argv[2]
oracle._LIBPATH = os.path.join(sys.argv[2], "liboracle.so")
import pytest
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu and not slow",
                      *sys.argv[3:]]))
"""


# For the Python module the child loads the copy under the module's own name before the pins
# import it.
CHILD_EXACT = """
import importlib.util, sys
sys.path.insert(0, {root!r})
import oracle
spec = importlib.util.spec_from_file_location("oracle.exact_riemann_general", sys.argv[1])
mod = importlib.util.module_from_spec(spec)
sys.modules[spec.name] = mod
spec.loader.exec_module(mod)
oracle.exact_riemann_general = mod
import pytest
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu and not slow",
                      *sys.argv[2:]]))
"""


def _run(tmp, k, kind, text):
    d = os.path.join(tmp, f"case{k:02d}")
    os.makedirs(d)
    if kind == "c":
        src = os.path.join(d, "dgsrhd_oracle.c")
        argv = [CHILD.format(root=ROOT), src, os.path.join(d, "_build"), *PINS]
    else:
        src = os.path.join(d, "exact_riemann_general.py")
        argv = [CHILD_EXACT.format(root=ROOT), src, *EXACT_PINS]
    with open(src, "w") as f:
        f.write(text)
    proc = subprocess.run([sys.executable, "-c", *argv], cwd=ROOT, capture_output=True,
                          text=True, timeout=600)
    return proc.returncode, (proc.stdout + proc.stderr)[-1500:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    tmp = str(tmp_path_factory.mktemp("planted"))
    jobs = {}
    for kind, path, mutations in (("c", SOURCE, MUTATIONS), ("py", EXACT_SOURCE, EXACT_MUTATIONS)):
        original = open(path).read()
        jobs[f"unmodified {kind}"] = (kind, original)
        for name, old, new in mutations:
            assert original.count(old) == 1, f"{name}: the text to replace must occur exactly once"
            jobs[name] = (kind, original.replace(old, new))
    with ThreadPoolExecutor(max_workers=max(1, min(6, (os.cpu_count() or 2) - 1))) as ex:
        futures = {name: ex.submit(_run, tmp, k, kind, text)
                   for k, (name, (kind, text)) in enumerate(jobs.items())}
        return {name: fut.result() for name, fut in futures.items()}


@pytest.mark.parametrize("kind", ["c", "py"])
def test_unmodified_copy_passes_the_pins(outcomes, kind):
    rc, tail = outcomes[f"unmodified {kind}"]
    assert rc == 0, tail


@pytest.mark.parametrize("name", [m[0] for m in MUTATIONS + EXACT_MUTATIONS])
def test_planted_mistake_fails_a_pin(outcomes, name):
    rc, tail = outcomes[name]
    # pytest's exit code 1: tests ran and some failed (not a crash or a collection error)
    assert rc == 1, f"{name}: exit {rc}\n{tail}"
