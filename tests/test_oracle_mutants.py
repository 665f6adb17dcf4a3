"""CPU test: plant plausible mistakes in copies of the oracle and check that
the pins catch every one.

Each mutant is the oracle source with one textual change (a dropped term, a
wrong sign, a wrong index, a transposed operand, the other reading of eq. 4),
compiled into a temporary directory; the committed oracle is never touched.
"""
import os
import subprocess

import pytest

import oracle
import oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "gp_oracle.c")

MUTANTS = {
    "corr_ignores_p": ("return exp(-theta * pow(a, p));", "return exp(-theta * pow(a, 2.0));"),
    "corr_wrong_index": ("gpo_corr_1d(xi[k] - xj[k], theta[k], p, fam)", "gpo_corr_1d(xi[k] - xj[0], theta[k], p, fam)"),
    "corr_sign": ("return exp(-theta * pow(a, p));", "return exp(theta * pow(a, p));"),
    "matern12_squares": ("if (fam == GPO_MATERN12) return exp(-theta * a);",
                         "if (fam == GPO_MATERN12) return exp(-theta * a * a);"),
    "matern32_constant": ("real h = sqrt((real)3) * theta * a;", "real h = sqrt((real)5) * theta * a;"),
    "matern32_linear_coeff": ("return (1.0 + h) * exp(-h);", "return (1.0 + 0.5 * h) * exp(-h);"),
    "q_zero_threshold_off": ("return Q <= 16.0 * n * u * u * bb;", "return Q <= 0.0;"),
    "predict_nugget_ignored": ("real c0 = nugget_in_var ? 1.0 + delta : 1.0;", "real c0 = 1.0;"),
    "matern52_drops_quadratic": ("return (1.0 + h + h * h / 3.0) * exp(-h);", "return (1.0 + h) * exp(-h);"),
    "matern52_quadratic_coeff": ("return (1.0 + h + h * h / 3.0) * exp(-h);",
                                 "return (1.0 + h + h * h / 2.0) * exp(-h);"),
    "nugget_everywhere": ("if (i == j) v += delta;", "v += delta;"),
    "nugget_dropped": ("if (i == j) v += delta;", ";"),
    "chol_update_sign": ("s -= L[(size_t)i * n + k] * L[(size_t)j * n + k];",
                         "s += L[(size_t)i * n + k] * L[(size_t)j * n + k];"),
    "chol_offdiag_mul": ("L[(size_t)i * n + j] = s / L[(size_t)j * n + j];",
                         "L[(size_t)i * n + j] = s * L[(size_t)j * n + j];"),
    "forward_transposed": ("for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * z[k];",
                           "for (int k = 0; k < i; ++k) s -= L[(size_t)k * n + i] * z[k];"),
    "backward_transposed": ("for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * w[k];",
                            "for (int k = i + 1; k < n; ++k) s -= L[(size_t)i * n + k] * w[k];"),
    "mu_inverted": ("real mu = ab / aa;\n    real Q = 0.0, bb", "real mu = aa / ab;\n    real Q = 0.0, bb"),
    "residual_sign": ("e[i] = b[i] - mu * a[i]; Q += e[i] * e[i]; bb", "e[i] = b[i] + mu * a[i]; Q += e[i] * e[i]; bb"),
    "logdet_not_doubled": ("    logdet *= 2.0;\n    real sigma2", "    real sigma2"),
    "nll_uses_sigma2": ("out[0] = logdet + n * log(Q);", "out[0] = logdet + n * log(Q / n);"),
    "nll_drops_n": ("out[0] = logdet + n * log(Q);", "out[0] = logdet + log(Q);"),
    "sigma2_not_over_n": ("real sigma2 = Q / n;\n    out[1]", "real sigma2 = Q;\n    out[1]"),
    "predict_drops_mu": ("yhat[m] = mu + yh;", "yhat[m] = yh;"),
    "predict_var_sign": ("s2[m] = sigma2 * (c0 - vv + g * g / aa);", "s2[m] = sigma2 * (c0 + vv + g * g / aa);"),
    "predict_var_unsquared": ("s2[m] = sigma2 * (c0 - vv + g * g / aa);", "s2[m] = sigma2 * (c0 - vv + g / aa);"),
    "predict_nugget_in_r": ("gpo_corr_pair(d, xs, x + (size_t)i * d, theta, p, fam);",
                            "gpo_corr_pair(d, xs, x + (size_t)i * d, theta, p, fam) + 1e-6;"),
    "cond_no_anorm": ("return anorm * est;", "return est;"),
    "cond_start_unscaled": ("for (int i = 0; i < n; ++i) v[i] = 1.0 / n;", "for (int i = 0; i < n; ++i) v[i] = 1.0;"),
    "cond_est_not_abs": ("for (int i = 0; i < n; ++i) est += fabs(yv[i]);", "for (int i = 0; i < n; ++i) est += yv[i];"),
    "cond_no_second_round": ("if (zmax <= ztv || jmax == jprev) break;", "break;"),
    "grad_trace_sign": ("tr += Ri[(size_t)j * n + i] * dR;", "tr -= Ri[(size_t)j * n + i] * dR;"),
    "grad_drops_n_over_q": ("grad[k] = tr - n / Q * quad;", "grad[k] = tr - quad;"),
    "grad_power_wrong": ("    return -pow(a, p);", "    return -pow(a, p - 1.0);"),
    "grad_matern32_dlog": ("return -h / (1.0 + h) * sqrt((real)3) * a;", "return -h * sqrt((real)3) * a;"),
    "grad_matern52_dlog": ("return -h * (1.0 + h) / (3.0 * (1.0 + h + h * h / 3.0)) * sqrt((real)5) * a;",
                           "return -h * (1.0 + h) / (3.0 * (1.0 + h + h * h / 3.0)) * sqrt((real)3) * a;"),
    "grad_quad_one_sided": ("quad += w[i] * dR * w[j];", "quad += w[i] * dR * w[i];"),
    "grad_exponential_dlog": ("if (fam == GPO_MATERN12) return -a;", "if (fam == GPO_MATERN12) return -a * a;"),
}


def _build_mutant(tmpdir, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mutated = src.replace(old, new, 1)
    cpath = os.path.join(tmpdir, f"m_{name}.c")
    lib = os.path.join(tmpdir, f"libm_{name}.so")
    with open(cpath, "w") as f:
        f.write(mutated)
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                    "-D_DEFAULT_SOURCE", cpath, "-o", lib, "-lm"], check=True)
    return oracle.Oracle(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    orc = _build_mutant(str(tmp_path), name, old, new)
    failed = []
    for check in pins.ALL_CHECKS:
        try:
            check(orc)
        except Exception as exc:  # AssertionError, or a numeric error from nonsense output
            failed.append((check.__name__, type(exc).__name__))
    assert failed, f"no pin caught mutant {name}"
