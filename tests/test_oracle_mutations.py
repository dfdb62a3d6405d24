"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle -- its C source, its
Python driver or the FE oracle -- and runs the oracle's pin tests against that
copy; they must fail.  An unmodified copy must pass, so a failure is the planted
mistake's, and every mutant must compile, so a build error is not counted as a
catch.  The copies live in temporary trees that mirror the repository: the
patched oracle/, the pin tests with their golden fixture, and the input
generators.
"""
import os
import re
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_TESTS = ["test_oracle_pins.py", "test_oracle_compression.py", "test_oracle_grad.py",
             "test_oracle_predictor.py", "test_fe_oracle.py"]

# (id, file under oracle/, text, replacement, the passage the mistake contradicts)
MUTATIONS = [
    ("fractions_swapped", "dmn_oracle.c", "(s < 0) ? -t->c2[j] : t->c1[j]", "(s < 0) ? -t->c1[j] : t->c2[j]",
     "gradient operator: the left subtree's block is -c2 N, the right one's +c1 N (Sec. 3.1)"),
    ("sym_factor", "dmn_oracle.c", "T[r][c] = 0.5 * (((r == m)", "T[r][c] = (((r == m)",
     "N a = sym(a (x) n) (Sec. 3.1)"),
    ("spherical_normal", "dmn_oracle.c", "nrm[j][1] = sin(al) * sin(be);", "nrm[j][1] = cos(al) * sin(be);",
     "n = (sin a cos b, sin a sin b, cos a) (Sec. 2.3)"),
    ("barycentric_system", "dmn_oracle.c", "{0.0, 1.0 / 3.0, 0.5, lam2}", "{0.0, 1.0 / 3.0, 1.0, lam2}",
     "corners UD, ISO, PI of the orientation triangle (Sec. 2.3)"),
    ("quadratic_shape_functions", "dmn_oracle.c", "ph[3] = 4.0 * v[0] * v[1]; ph[4] = 4.0 * v[0] * v[2];",
     "ph[3] = 4.0 * v[0] * v[2]; ph[4] = 4.0 * v[0] * v[1];", "quadratic shape functions (Sec. 2.3)"),
    ("yield_factor", "dmn_oracle.c", "double f = ns - sqrt(2.0 / 3.0) * sy;", "double f = ns - sy;",
     "von Mises yield function (Sec. 4.1)"),
    ("hardening_factor", "dmn_oracle.c", "dg = f / (2.0 * G + 2.0 * ph->H / 3.0);", "dg = f / (2.0 * G + ph->H / 3.0);",
     "radial return with linear hardening (Sec. 4.1)"),
    ("tangent_theta_bar_sign", "dmn_oracle.c", "double thb = 1.0 / (1.0 + Hp / (3.0 * G)) - (1.0 - th);",
     "double thb = 1.0 / (1.0 + Hp / (3.0 * G)) + (1.0 - th);", "consistent J2 tangent (Sec. 4.1)"),
    ("hardening_slope_in_tangent", "dmn_oracle.c", "    Hp = ph->H;\n", "    Hp = 0.0;\n",
     "consistent J2 tangent with the hardening slope (Sec. 4.1)"),
    ("equivalent_plastic_strain", "dmn_oracle.c", "z_new[0] = ab_n + sqrt(2.0 / 3.0) * dg;", "z_new[0] = ab_n + dg;",
     "equivalent plastic strain of the hardening law (Sec. 4.1)"),
    ("exp_linear_rate", "dmn_oracle.c", "double e = exp(-r * ab);", "double e = exp(-ab);",
     "exponential-linear hardening (Sec. 4.1)"),
    ("effective_stress_weights", "dmn_oracle.c", "ws->sbar[I] += t->w[l] * ws->sig[l][I];",
     "ws->sbar[I] += ws->sig[l][I] / t->L;", "effective stress as the weighted leaf average (Sec. 3.2)"),
    ("cholesky_diagonal_term", "dmn_oracle.c",
     "for (int b = 0; b < a; ++b) { double v = LL(c, 3 * cn + b); s -= v * v; }", "",
     "Newton step J da = -R by Cholesky factorisation (Sec. 4.6)"),
    ("back_substitution_term", "dmn_oracle.c",
     "for (int b = a + 1; b < 3; ++b) s -= LL(3 * cn + b, c) * x[3 * cn + b];", "",
     "Newton step J da = -R by Cholesky factorisation (Sec. 4.6)"),
    ("tangent_rhs_sign", "dmn_oracle.c", "x[3 * t->cidx[j] + m] -= c * s;", "x[3 * t->cidx[j] + m] += c * s;",
     "algorithmic tangent from the six-right-hand-side system (Sec. 3.2)"),
    ("rotation_transposed", "dmn_oracle.c",
     "s += to_local ? Q[a * 3 + i] * T[a][b] * Q[b * 3 + j] : Q[i * 3 + a] * T[a][b] * Q[j * 3 + b];",
     "s += to_local ? Q[i * 3 + a] * T[a][b] * Q[j * 3 + b] : Q[a * 3 + i] * T[a][b] * Q[b * 3 + j];",
     "material frame from the eigenvectors of A2 (Sec. 5)"),
    ("mandel_weight", "dmn_oracle.c", "static double mweight(int I) { return I < 3 ? 1.0 : R2; }",
     "static double mweight(int I) { return I < 3 ? 1.0 : 2.0; }", "Mandel notation of the rotated stiffness"),
    ("stopping_tolerance", "dmn_oracle.c", "if (rn <= t->tol * (double)N * mandel_norm(ws->sbar)) break;",
     "if (rn <= 1e4 * t->tol * (double)N * mandel_norm(ws->sbar)) break;", "stopping criterion (Sec. 4.6)"),
    ("compression_keeps_pass_through", "dmn_oracle.c", "t->cidx[j] = (wl > 0.0 && wr > 0.0) ? 0 : -1;",
     "t->cidx[j] = (wl > 0.0 || wr > 0.0) ? 0 : -1;", "compression removes laminates with a weightless side (Sec. 3.1)"),
    ("dual_sine_rule", "dmn_oracle.c", "return dn(sin(a.v), cos(a.v) * a.d);", "return dn(sin(a.v), -cos(a.v) * a.d);",
     "derivative of the spherical normal in the angles (Sec. 2.3)"),
    ("dual_product_rule", "dmn_oracle.c", "return dn(a.v * b.v, a.d * b.v + a.v * b.d);", "return dn(a.v * b.v, a.d * b.v);",
     "exact partial derivatives of R and sigma_bar (Sec. 3.2)"),
    ("dual_quotient_rule", "dmn_oracle.c", "(a.d * b.v - a.v * b.d) / (b.v * b.v)", "a.d / b.v",
     "exact partial derivatives of R and sigma_bar (Sec. 3.2)"),
    ("dual_weight_normalisation", "dmn_oracle.c", "u->wn[l] = d_div(dn(w_raw[l], dw[l]), sw);",
     "u->wn[l] = d_div(dn(w_raw[l], dw[l]), dc(sw.v));", "weights normalised to sum 1 (Sec. 2.1)"),
    ("dual_fraction_complement", "dmn_oracle.c", "u->c2[j] = d_sub(dc(1.0), u->c1[j]);",
     "u->c2[j] = dn(1.0 - u->c1[j].v, u->c1[j].d);", "c2 = 1 - c1 (Sec. 2.1)"),
    ("dual_hardening_exponential", "dmn_oracle.c", "dual e = d_exp(d_scale(-r, ab));", "dual e = dc(exp(-r * ab.v));",
     "exponential-linear hardening (Sec. 4.1)"),
    ("dual_tangent_solve_term", "dmn_oracle.c", "      dx[r] -= s;\n", "      dx[r] -= 0.0 * s;\n",
     "derivative of the six-right-hand-side solve of Eq. (lin_system_da_dE)"),
    ("adjoint_solve_missing", "dmn_oracle.c", "    chol_solve(&t, ws, lam);\n", "",
     "implicit-function gradient: J lam = (d sigma_bar/da)^T g (Sec. 3.2)"),
    ("adjoint_sign", "dmn_oracle.c", "for (int r = 0; r < n; ++r) v -= lam[r] * u->R[r].d;",
     "for (int r = 0; r < n; ++r) v += lam[r] * u->R[r].d;", "implicit-function gradient (Sec. 3.2)"),
    ("extrapolation_sign", "__init__.py", "start[S0 - J:] = a_n + rho[None, :] * change",
     "start[S0 - J:] = a_n - rho[None, :] * change", "extrapolated start a^n + rho (a^n - a^(n-1))"),
    ("extrapolation_clip", "__init__.py", "np.clip(r, 0.0, 1.0)", "np.clip(r, 0.0, 2.0)",
     "extrapolation factor clipped to at most 1 (a factor below 0 is never used: only rho > 0 extrapolates)"),
    ("restart_disabled", "__init__.py", "if fail.size:", "if False:", "restart from a^n after a failed extrapolation"),
    ("fe_shear_factor", "fe_oracle.py", "s = 1.0 / math.sqrt(2.0)", "s = 0.5", "Mandel shear strain of sym(grad u)"),
    ("fe_shape_derivative", "fe_oracle.py", "out[a, 1] = NODE_SIGNS[a, 1] * f[0] * f[2] / 8.0",
     "out[a, 1] = NODE_SIGNS[a, 1] * f[0] * f[1] / 8.0", "trilinear shape functions"),
    ("fe_jacobian_transposed", "fe_oracle.py", "dNdx = dN[g] @ np.linalg.inv(J)", "dNdx = dN[g] @ np.linalg.inv(J).T",
     "isoparametric map of the hexahedron"),
]


def _mirror(dest, mutation):
    """A tree with the (patched) oracle, the pin tests and the input generators; returns None or an error."""
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dest, "oracle"),
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    os.symlink(os.path.join(ROOT, "paper_2103_08253_gb300"), os.path.join(dest, "paper_2103_08253_gb300"))
    os.makedirs(os.path.join(dest, "tests"))
    for f in ["conftest.py"] + PIN_TESTS:
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dest, "tests", f))
    os.symlink(os.path.join(ROOT, "tests", "golden"), os.path.join(dest, "tests", "golden"))
    if mutation is not None:
        _, fname, text, repl, _ = mutation
        path = os.path.join(dest, "oracle", fname)
        src = open(path).read()
        if src.count(text) != 1:
            return "the text to replace occurs %d times in %s" % (src.count(text), fname)
        open(path, "w").write(src.replace(text, repl))
    # compile the C oracle here, so that a mutant that does not build is not mistaken for a catch
    os.makedirs(os.path.join(dest, "oracle", "_build"))
    r = subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o",
                        os.path.join(dest, "oracle", "_build", "liboracle_dmn.so"),
                        os.path.join(dest, "oracle", "dmn_oracle.c"), "-lm"], capture_output=True, text=True)
    return None if r.returncode == 0 else "does not compile: " + r.stderr[-500:]


def _run(dest, mutation):
    os.makedirs(dest)
    err = _mirror(dest, mutation)
    if err:
        return None, err
    env = dict(os.environ, OMP_NUM_THREADS="2", PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]
                       + ["tests/" + f for f in PIN_TESTS], cwd=dest, env=env, capture_output=True, text=True,
                       timeout=600)
    failed = re.findall(r"^FAILED (\S+)", r.stdout, re.M)
    return r.returncode, (failed[0] if failed else r.stdout[-1500:])


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    base = str(tmp_path_factory.mktemp("oracle_mutants"))
    jobs = [("control", None)] + [(m[0], m) for m in MUTATIONS]
    with ThreadPoolExecutor(max_workers=max(1, min(8, (os.cpu_count() or 2) // 2))) as ex:
        futures = {name: ex.submit(_run, os.path.join(base, name), m) for name, m in jobs}
        return {name: f.result() for name, f in futures.items()}


def test_unmodified_copy_passes_the_pins(outcomes):
    rc, info = outcomes["control"]
    assert rc == 0, info


@pytest.mark.parametrize("mutation", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(outcomes, mutation):
    rc, info = outcomes[mutation[0]]
    assert rc is not None, info               # the mutation applies and builds
    assert rc == 1, "not caught (%s): %s" % (mutation[4], info)
