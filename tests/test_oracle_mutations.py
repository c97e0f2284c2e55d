"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of oracle/cg_oracle.c (a flipped sign
in a local partial derivative, a dropped term, a wrong factor, a transposed
operand), builds it with gcc and runs the pin suites (the model pins and the
expression-interpreter pins) against it in a subprocess; at least one pin
must fail.  The real oracle is never modified.
"""
import os
import subprocess
import sys

import pytest

from tests.conftest import ROOT

SRC = os.path.join(ROOT, "oracle", "cg_oracle.c")

MUTATIONS = {
    # reverse sweep: d(a - b)/db = -1 -> +1
    "sub_partial_sign": ("return push(T, VAL(a) - VAL(b), a, 1.0, b, -1.0);",
                         "return push(T, VAL(a) - VAL(b), a, 1.0, b, 1.0);"),
    # d(a/b)/db = -q/b -> q/b
    "div_partial_sign": ("return push(T, q, a, 1.0 / VAL(b), b, -q / VAL(b));",
                         "return push(T, q, a, 1.0 / VAL(b), b, q / VAL(b));"),
    # d exp(x)/dx = e -> 1
    "exp_partial": ("double e = exp(VAL(a)); return push(T, e, a, e, -1, 0.0);",
                    "double e = exp(VAL(a)); return push(T, e, a, 1.0, -1, 0.0);"),
    # d erfc/dz sign
    "erfc_partial_sign": ("-2.0 / sqrt(M_PI) * exp(-z * z)", "2.0 / sqrt(M_PI) * exp(-z * z)"),
    # Gaussian width: 2 s^2 -> s^2
    "gauss_factor_two": ("int32_t den = t_mulc(T, t_mul(T, s, s), 2.0);  /* 2 s^2 */",
                         "int32_t den = t_mul(T, s, s);  /* 2 s^2 */"),
    # chi-square weight 1/max(y, 1) -> 1
    "chi2_weight": ("double w = 1.0 / fmax(y, 1.0);\n        int32_t r = t_rsubc(T, y, f);",
                    "double w = 1.0;\n        int32_t r = t_rsubc(T, y, f);"),
    # Baker-Cousins factor 2 dropped
    "bc_factor": ("return t_mulc(T, inner, 2.0);", "return inner;"),
    # mixture normalisation: Z_E = e^{-l lo} - e^{-l hi} -> only the first term
    "mixture_ZE": ("int32_t ZE = t_sub(&T, t_exp(&T, t_mulc(&T, lam, -lo)), t_exp(&T, t_mulc(&T, lam, -hi)));",
                   "int32_t ZE = t_exp(&T, t_mulc(&T, lam, -lo));"),
    # rotation: v = -s dx + c dy -> s dx + c dy
    "rotation_sign": ("int32_t v = t_add(&T, t_neg(&T, t_mul(&T, s, dx)), t_mul(&T, c, dy));",
                      "int32_t v = t_add(&T, t_mul(&T, s, dx), t_mul(&T, c, dy));"),
    # polynomial in t: (2x - lo - hi)/(hi - lo) -> (x - lo)/(hi - lo)
    "poly_t_map": ("double u = (poly_mode == 1) ? (2.0 * x - lo - hi) / (hi - lo) : x;\n        int32_t f = rec_gauss_poly(&T, K, D, x, u);\n        int32_t t = rec_binned_term",
                   "double u = (poly_mode == 1) ? (x - lo) / (hi - lo) : x;\n        int32_t f = rec_gauss_poly(&T, K, D, x, u);\n        int32_t t = rec_binned_term"),
    # Gauss-Newton diagonal: h J_k^2 -> h J_k
    "gn_diag_square": ("for (int32_t k = 0; k < P; ++k) nadd(&acc[k], hi_ * adj[k] * adj[k]);",
                       "for (int32_t k = 0; k < P; ++k) nadd(&acc[k], hi_ * adj[k]);"),
    # Gauss-Newton matrix: J_a J_b -> J_a J_a (the diagonal's product everywhere)
    "gnmat_transposed_factor": ("nadd(&acc[(size_t)a * P + b], hi_ * adj[a] * adj[b]);",
                                "nadd(&acc[(size_t)a * P + b], hi_ * adj[a] * adj[a]);"),
    # Gauss-Newton matrix: Poisson curvature y/f^2 -> y/f
    "gnmat_poisson_curvature": ("else if (obj == OBJ_POISSON) hi_ = (y[i] > 0.0) ? y[i] / (fv * fv) : 0.0;\n        else hi_ = (y[i] > 0.0) ? 2.0 * y[i] / (fv * fv) : 0.0;\n        for (int32_t a",
                                "else if (obj == OBJ_POISSON) hi_ = (y[i] > 0.0) ? y[i] / fv : 0.0;\n        else hi_ = (y[i] > 0.0) ? 2.0 * y[i] / (fv * fv) : 0.0;\n        for (int32_t a"),
    # expression interpreter: d sqrt(a)/da = 1/(2 sqrt a) -> 1/sqrt a
    "expr_sqrt_partial": ("return push(T, r, a, 0.5 / r, -1, 0.0);", "return push(T, r, a, 1.0 / r, -1, 0.0);"),
    # expression interpreter: d a^k/da = k a^(k-1) -> k a^k
    "expr_powi_partial": ("(double)k * pow(x, (double)(k - 1))", "(double)k * pow(x, (double)k)"),
    # expression interpreter: max sends its adjoint to the smaller operand
    "expr_max_branch": ("if (VAL(a) >= VAL(b)) return push(T, VAL(a), a, 1.0, b, 0.0);",
                        "if (VAL(a) >= VAL(b)) return push(T, VAL(a), a, 0.0, b, 1.0);"),
    # expression interpreter: the element index off by one
    "expr_index": ("case 3: t[j] = t_const(&T, (double)e); break;", "case 3: t[j] = t_const(&T, (double)(e + 1)); break;"),
    # compensated sum loses its correction
    "neumaier_dropped": ("static double nval(const nsum *acc) { return acc->s + acc->c; }",
                         "static double nval(const nsum *acc) { return acc->s; }"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor not found: " + name
    msrc = tmp_path / "cg_oracle_mut.c"
    msrc.write_text(src.replace(old, new))
    lib = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(lib),
                           str(msrc), "-lm"])
    env = dict(os.environ, CG_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_expr_cpu.py")], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "no pin failed for mutation %s:\n%s" % (name, r.stdout[-2000:])


# Planted mistakes in copies of the fit drivers (oracle/fit.py), each caught
# by the drivers' closed-form pins.
FIT_SRC = os.path.join(ROOT, "oracle", "fit.py")
FIT_MUTATIONS = {
    # BFGS inverse update with the outer products transposed
    "bfgs_update_transposed": ("H = (I - r * np.outer(s, y)) @ H @ (I - r * np.outer(y, s)) + r * np.outer(s, s)",
                               "H = (I - r * np.outer(y, s)) @ H @ (I - r * np.outer(s, y)) + r * np.outer(s, s)",
                               "check_bfgs_secant"),
    # initial inverse Hessian = GN instead of 1 / GN
    "bfgs_h0_not_inverted": ("Hdiag = np.where(d0 > 0, 1.0 / np.where(d0 > 0, d0, 1.0), 1.0)",
                             "Hdiag = np.where(d0 > 0, np.where(d0 > 0, d0, 1.0), 1.0)",
                             "check_bfgs_first_step_is_newton"),
    # damping relaxed by 2 instead of 10 after an accepted step
    "lm_damping_factor": ("lam = max(lam * 0.1, 1e-12)", "lam = max(lam * 0.5, 1e-12)",
                          "check_lm_steps_on_a_separable_quadratic"),
    # step towards larger F
    "lm_step_sign": ("delta = _chol_solve(G + lam * np.diag(dpos), -g)", "delta = _chol_solve(G + lam * np.diag(dpos), g)",
                     "check_lm_steps_on_a_separable_quadratic"),
}


@pytest.mark.parametrize("name", sorted(FIT_MUTATIONS))
def test_fit_pins_catch_mutation(name):
    import types
    import oracle.fit as real
    from tests import test_oracle_pins as pins
    old, new, check = FIT_MUTATIONS[name]
    src = open(FIT_SRC).read()
    assert src.count(old) == 1, "mutation anchor not found: " + name
    mod = types.ModuleType("fit_mutated")
    exec(compile(src.replace(old, new), "fit_mutated", "exec"), mod.__dict__)
    which = "lm_fit" if check.startswith("check_lm") else "bfgs_fit"
    getattr(pins, check)(getattr(real, which))          # the real driver passes
    with pytest.raises(AssertionError):
        getattr(pins, check)(getattr(mod, which))       # the planted mistake does not
