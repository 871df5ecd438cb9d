"""The oracle pins must catch plausible mistakes.

Each case below plants one mistake in a private copy of the oracle's C
source (a dropped term, a flipped sign, a wrong slice weight, a missing
diagonal, rounding instead of truncation, an off-by-one exponent, a wrong
slice index, a missing absolute value, a dropped Dot2 correction; for the
mod2as oracle a skipped last row, a wrong column, a dropped first term),
compiles it, and runs the matching pins (tests/test_oracle_pins.py or
tests/test_oracle_spmv_pins.py) against it in a subprocess: every mutant
must make its suite fail.  Nothing here touches a GPU.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mxm_oracle.c")

MUTANTS = {
    "naive_drops_last_term": (
        "for (int64_t l = 0; l < k; ++l) s += A[i * k + l] * B[l * n + j];\n      C[i * n + j] = s;\n    }\n  }\n}\n\n/* arbb_mxm2a",
        "for (int64_t l = 0; l + 1 < k; ++l) s += A[i * k + l] * B[l * n + j];\n      C[i * n + j] = s;\n    }\n  }\n}\n\n/* arbb_mxm2a"),
    "naive_sign_flip": (
        "s += A[i * k + l] * B[l * n + j];\n      C[i * n + j] = s;\n    }\n  }\n}\n\n/* arbb_mxm2a",
        "s -= A[i * k + l] * B[l * n + j];\n      C[i * n + j] = s;\n    }\n  }\n}\n\n/* arbb_mxm2a"),
    "dot2_drops_correction": ("s = s + (q + r);\n  }\n  return p + s;",
                              "s = s + q;\n  }\n  return p + s;"),
    "ozaki_wrong_weight": (
        "acc = acc + ldexp((double)Dg, -beta * g);\n  }\n  return ldexp(acc, e_i + f_j);",
        "acc = acc + ldexp((double)Dg, -beta * (g - 1));\n  }\n  return ldexp(acc, e_i + f_j);"),
    "ozaki_drops_last_diagonal": (
        "double acc = 0.0;\n  for (int g = S + 1; g >= 2; --g) {\n    int64_t Dg = 0;\n    for (int s = 1; s <= g - 1; ++s) {\n      int t = g - s;",
        "double acc = 0.0;\n  for (int g = S; g >= 2; --g) {\n    int64_t Dg = 0;\n    for (int s = 1; s <= g - 1; ++s) {\n      int t = g - s;"),
    "ozaki_rounds_not_truncates": ("double q = trunc(t);", "double q = round(t);"),
    "ozaki_exponent_off_by_one": ("(void)frexp(x, &e);\n  return e;", "(void)frexp(x, &e);\n  return e + 1;"),
    "ozaki_wrong_slice_index": (
        "const int16_t* b = dBt + (int64_t)(t - 1) * planeB + j * k;",
        "const int16_t* b = dBt + (int64_t)(s - 1) * planeB + j * k; (void)t;"),
    "abs_missing_fabs": (
        "s += fabs(A[i * k + l]) * fabs(B[l * n + j]);\n      C[i * n + j] = s;",
        "s += A[i * k + l] * fabs(B[l * n + j]);\n      C[i * n + j] = s;"),
    # mod2as (Sec. 3.2); checked by tests/test_oracle_spmv_pins.py
    "spmv_skips_last_row": (
        "for (i = 0; i < nrows; ++i) {\n    double t = 0.0;\n    for (int64_t j = rowp[i]; j < rowp[i + 1]; ++j) t = t + vals[j] * x[indx[j]];",
        "for (i = 0; i < nrows - 1; ++i) {\n    double t = 0.0;\n    for (int64_t j = rowp[i]; j < rowp[i + 1]; ++j) t = t + vals[j] * x[indx[j]];"),
    "spmv_wrong_column": ("t = t + vals[j] * x[indx[j]];", "t = t + vals[j] * x[j % ncols];"),
    "spmv_drops_first_term": (
        "for (int64_t j = rowp[i]; j < rowp[i + 1]; ++j) t = t + vals[j] * x[indx[j]];",
        "for (int64_t j = rowp[i] + 1; j < rowp[i + 1]; ++j) t = t + vals[j] * x[indx[j]];"),
    "spmv_dot2_drops_correction": ("s = s + (q + r);\n    }\n    y[i] = p + s;",
                                   "s = s + q;\n    }\n    y[i] = p + s;"),
    "spmv_abs_missing_fabs": ("t = t + fabs(vals[j]) * fabs(x[indx[j]]);",
                              "t = t + vals[j] * fabs(x[indx[j]]);"),
    # conjugate gradients (Sec. 3.4); checked by tests/test_oracle_cg_pins.py
    "cg_beta_inverted": ("const double beta = r2 / r2_old;", "const double beta = r2_old / r2;"),
    "cg_residual_sign": ("r[i] = r[i] - alpha * q[i];", "r[i] = r[i] + alpha * q[i];"),
    "cg_direction_from_residual": ("p[i] = r[i] + beta * p[i];", "p[i] = r[i] + beta * r[i];"),
    "cg_x_along_residual": ("x[i] = x[i] + alpha * p[i];", "x[i] = x[i] + alpha * r[i];"),
    "cg_no_beta": ("p[i] = r[i] + beta * p[i];", "p[i] = r[i] + 0.0 * beta * p[i];"),
    "cg_product_drops_diagonal": ("t = t + vals[j] * p[indx[j]];",
                                  "if (indx[j] != i) t = t + vals[j] * p[indx[j]];"),
    "cg_stop_off_by_one": ("while (r2 > stop && k < max_iters) {",
                           "while (r2 > stop && k <= max_iters) {"),
    # mod2f (Sec. 3.3); checked by tests/test_oracle_fft_pins.py
    "fft_twiddle_sign": ("  *s = -sin(ang);", "  *s = sin(ang);"),
    "fft_twiddle_index": ("        twiddle(n, L, &c, &s);", "        twiddle(n + 1, L, &c, &s);"),
    "fft_difference_sign": ("const double dr = ar - br, di = ai - bi;",
                            "const double dr = br - ar, di = bi - ai;"),
    "fft_no_bit_reversal": ("    F[2 * r] = w[2 * p];\n    F[2 * r + 1] = w[2 * p + 1];",
                            "    F[2 * p] = w[2 * p]; (void)r;\n    F[2 * p + 1] = w[2 * p + 1];"),
    "fft_complex_product": ("x1[1] = dr * s + di * c;", "x1[1] = dr * s - di * c;"),
    "dft_conjugated_term": ("im = im + (a * s + b * c);", "im = im + (a * s - b * c);"),
    # the balanced 8-bit digit split; checked by tests/test_oracle_rn8_pins.py
    "rn8_truncates": ("int64_t V = (int64_t)nearbyint(ldexp(x, 8 * S - e1));",
                      "int64_t V = (int64_t)trunc(ldexp(x, 8 * S - e1));"),
    "rn8_unbalanced_digits": ("const int64_t dig = r >= 128 ? r - 256 : r;",
                              "const int64_t dig = r;"),
    "rn8_no_exponent_offset": ("    for (int64_t i = 0; i < cnt; ++i) exps[i] += 1;",
                               "    for (int64_t i = 0; i < cnt; ++i) exps[i] += 0;"),
    "rn8_digit_order": ("    d[(s - 1) * stride] = (int16_t)dig;", "    d[(S - s) * stride] = (int16_t)dig;"),
}
PINS = {name: "test_oracle_spmv_pins.py" for name in MUTANTS if name.startswith("spmv_")}
PINS.update({name: "test_oracle_cg_pins.py" for name in MUTANTS if name.startswith("cg_")})
PINS.update({name: "test_oracle_fft_pins.py" for name in MUTANTS
             if name.startswith(("fft_", "dft_"))})
PINS.update({name: "test_oracle_rn8_pins.py" for name in MUTANTS if name.startswith("rn8_")})


def _compile(src_text, out_dir):
    c = os.path.join(out_dir, "mut.c")
    so = os.path.join(out_dir, "libmut.so")
    with open(c, "w") as fh:
        fh.write(src_text)
    cmd = ["gcc", "-std=c11", "-O2", "-fno-fast-math", "-ffp-contract=off", "-shared",
           "-fPIC", c, "-o", so, "-lm"]
    subprocess.run(cmd, check=True, capture_output=True)
    return so


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site for {name} not unique/found"
    so = _compile(text.replace(old, new), str(tmp_path))
    env = dict(os.environ, MXM_ORACLE_LIB=so, OMP_NUM_THREADS="2")
    pins = PINS.get(name, "test_oracle_pins.py")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pins)],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the oracle pins"
