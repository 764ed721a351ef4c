"""Plant plausible mistakes in a copy of the oracle and check a pin catches each one.

Each mutant is the oracle source with one textual edit, compiled to a
temporary library on the CPU.  The pins of ``pins.py`` must reject every
mutant; a mutant that survives would mean that part of the oracle is not
pinned to anything outside itself.
"""
import os
import subprocess

import pytest

import oracle
import pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "iht_oracle.c")

MUTANTS = {
    "bit_order_reversed": [("(2 * (i & 3))) & 3", "(2 * (3 - (i & 3)))) & 3")],
    "missing_as_dosage_0": [("default: return -1;", "default: return 0;")],
    "het_homalt_swapped": [("case 2: return 1;", "case 2: return 2;"),
                           ("case 3: return 2;", "case 3: return 1;")],
    "variance_denominator_n": [("/ (n_obs - 1.0)", "/ n_obs")],
    "no_centring": [("return v[j] * ((double)x - u[j]);", "return v[j] * (double)x;")],
    "no_scaling": [("return v[j] * ((double)x - u[j]);", "return ((double)x - u[j]);")],
    "counts_ignore_row_subset": [("cnt[bed_code(body, row_bytes, j, row_of(rows, a))]++",
                                  "cnt[bed_code(body, row_bytes, j, a)]++")],
    "tie_break_high_index": [("if (fa < fb) return 1;\n    return (a > b) - (a < b);",
                              "if (fa < fb) return 1;\n    return (a < b) - (a > b);")],
    "topk_smallest": [("if (fa > fb) return -1;\n    if (fa < fb) return 1;",
                       "if (fa > fb) return 1;\n    if (fa < fb) return -1;")],
    "step_not_squared": [("mu = num / den;", "mu = sqrt(num / den);")],
    "backtrack_test_reversed": [("if (mu < omega || bt", "if (mu > omega || bt")],
    "residual_sign": [("r[a] = y[a] - zv[a];", "r[a] = y[a] + zv[a];")],
    "no_step_shrink": [("mu /= opt->kappa;", "mu *= 1.0;")],
    "omega_without_1_minus_c": [("omega = (1.0 - opt->c) * dd / zz;", "omega = dd / zz;")],
    "omega_with_1_plus_c": [("omega = (1.0 - opt->c) * dd / zz;",
                             "omega = (1.0 + opt->c) * dd / zz;")],
    "convergence_without_plus_one": [("double step = sqrt(dn) / (sqrt(bn) + 1.0);",
                                      "double step = sqrt(dn);")],
    "convergence_plain_relative": [("double step = sqrt(dn) / (sqrt(bn) + 1.0);",
                                    "double step = sqrt(dn) / sqrt(bn);")],
    "htp_without_refit": [("if (htp) {\n            refit_ls(", "if (0) {\n            refit_ls(")],
    "htp_step_over_support": [("stepset = gam;", "stepset = S;")],
    "htp_refit_without_dependence_threshold": [("d > 1e-10 * gij ? sqrt(d) : 0.0", "d > 0.0 ? sqrt(d) : 0.0")],
    "covariates_not_scaled": [("return D->cv[t] * (D->cov[t * D->n + row_of(D->rows, a)] - D->cu[t]);",
                               "return (D->cov[t * D->n + row_of(D->rows, a)] - D->cu[t]);")],
    "covariate_variance_over_n": [("const double var = ss / (double)(n_rows - 1);",
                                   "const double var = ss / (double)n_rows;")],
    "covariates_ignore_row_subset": [("m += c[row_of(rows, a)];", "m += c[a];")],
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    text = open(SRC).read()
    for old, new in MUTANTS[name]:
        assert old in text, f"mutation anchor missing: {old!r}"
        text = text.replace(old, new)
    src = tmp_path / "mutant.c"
    src.write_text(text)
    out = str(tmp_path / "libmutant.so")
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                           "-o", out, str(src), "-lm"])
    lib = oracle.load(out, build_first=False)
    caught = []
    for pin in pins.ALL_PINS:
        try:
            pin(lib)
        except (AssertionError, RuntimeError, ValueError, IndexError) as e:
            caught.append(pin.__name__)
    assert caught, f"mutant {name} passes every pin"
