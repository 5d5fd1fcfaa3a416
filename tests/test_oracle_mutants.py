"""Every plausible mistake planted in the oracle must be caught by at least one pin.

Each mutant is a one-line edit of a copy of ``oracle/ngdbf_oracle.c`` (a
dropped term, a wrong sign or index, a transposed operand, an off-by-one),
compiled into a temporary library; the pin battery of ``oracle_pins`` then
runs against it in a child process and must fail.
"""
import os
import subprocess
import sys

import pytest

import oracle as oracle_pkg

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

MUTANTS = [
    ("philox key word", "^ c1 ^ k0;", "^ c1 ^ k1;"),
    ("philox multiplier", "mul0 = 0xD2511F53u", "mul0 = 0xD2511F57u"),
    ("philox rounds", "round < 10;", "round < 9;"),
    ("icdf sign ignored", "return (r & 0x80000000u) ? -g : g;", "return g;"),
    ("icdf level exponent", "ldexp(8.0 + s + 0.5 + node[i], -(j + 5))", "ldexp(8.0 + s + 0.5 + node[i], -(j + 4))"),
    ("icdf sub-interval offset", "ldexp(8.0 + s + 0.5 + node[i]", "ldexp(8.0 + s + node[i]"),
    ("icdf sub-interval bits", "int s = (int)((a >> 28) & 7u);", "int s = (int)((a >> 27) & 7u);"),
    ("icdf centering", "float v = one_plus_f - 1.5f;", "float v = one_plus_f - 1.0f;"),
    ("icdf fraction bits", "((a >> 5) & 0x007FFFFFu)", "((a >> 4) & 0x007FFFFFu)"),
    ("chebyshev node", "const double node[4] = {0.5 * C1, 0.5 * C3, -0.5 * C3, -0.5 * C1};",
     "const double node[4] = {0.5 * C3, 0.5 * C1, -0.5 * C1, -0.5 * C3};"),
    ("chebyshev b3 sign", "double b3 = (d03 * C3 - d12 * C1) * 0.5;", "double b3 = (d03 * C3 + d12 * C1) * 0.5;"),
    ("chebyshev c1", "(float)(2.0 * b1 - 6.0 * b3);", "(float)(2.0 * b1 + 6.0 * b3);"),
    ("chebyshev c0", "(float)(b0 - b2);", "(float)(b0 + b2);"),
    ("horner order", "fmaf(fmaf(fmaf(c[3], v, c[2]), v, c[1]), v, c[0])", "fmaf(fmaf(fmaf(c[3], v, c[1]), v, c[2]), v, c[0])"),
    ("phi scale", "0.5 * erfc(-z * 0.70710678118654752)", "0.5 * erfc(-z * 1.4142135623730951)"),
    ("no newton in f64", "for (int it = 0; it < 2; ++it)\n        z -=", "for (int it = 0; it < 0; ++it)\n        z -="),
    ("gauss4 output order", "for (int i = 0; i < 4; ++i) z[i] = oracle_gauss_f32(r[i]);",
     "for (int i = 0; i < 4; ++i) z[i] = oracle_gauss_f32(r[3 - i]);"),
    ("counter transposed", "uint32_t ctr[4] = {g, t, (uint32_t)frame, (uint32_t)(frame >> 32)};\n    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};\n    uint32_t r[4];\n    oracle_philox4x32_10(ctr, key, r);\n    for (int i = 0; i < 4; ++i) z[i] = oracle_gauss_f32",
     "uint32_t ctr[4] = {t, g, (uint32_t)frame, (uint32_t)(frame >> 32)};\n    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};\n    uint32_t r[4];\n    oracle_philox4x32_10(ctr, key, r);\n    for (int i = 0; i < 4; ++i) z[i] = oracle_gauss_f32"),
    ("noise scale", "return (float)((double)eta * (double)sigma);", "return (float)((double)eta * (double)sigma * (double)sigma);"),
    ("metric sign", "float e = xy + ws;", "float e = xy - ws;"),
    ("metric reassociated", "float e = xy + ws;\n    return e + q;", "float e = ws + q;\n    return xy + e;"),
    ("metric drops w", "float ws = w * (float)S;", "float ws = (float)S;"),
    ("metric drops x", "float xy = x > 0 ? ys : -ys;", "float xy = ys;"),
    ("metric64 sign", "return (x > 0 ? ys : -ys) + w * (double)S + q;", "return (x > 0 ? ys : -ys) - w * (double)S + q;"),
    ("flip tie", "flip = E < X->thr32[u[k]];", "flip = E <= X->thr32[u[k]];"),
    ("flip direction", "flip = E < X->thr64[u[k]];", "flip = E > X->thr64[u[k]];"),
    ("adapt on flips", "else if (adapt) u[k] += 1;", "if (adapt) u[k] += 1;"),
    ("threshold power", "thr[u] = (float)((double)theta * p);", "thr[u] = (float)((double)theta * p * (double)lambda);"),
    ("quantizer saturation", "if (k > kmax) k = kmax;", ""),
    ("quantizer half level", "return s * (k + 0.5) * (2.0 * y_max / nq);", "return s * k * (2.0 * y_max / nq);"),
    ("smoothing start", "T - P->smooth_window > 0 ? T - P->smooth_window : 0", "T - P->smooth_window + 1 > 0 ? T - P->smooth_window + 1 : 0"),
    ("smoothing tie", "(Xs[k] < 0 ? -1 : x[k])", "(Xs[k] < 0 ? -1 : 1)"),
    ("smoothing skips x(T)", "if (t >= t_smooth)\n", "if (t >= t_smooth && t < T)\n"),
    ("no final test", "for (int32_t t = 0; t <= T; ++t) {", "for (int32_t t = 0; t < T; ++t) {"),
    ("iteration count", "*iters = t;", "*iters = t + 1;"),
    ("sign of zero", "x[k] = v >= 0.0f ? 1 : -1;", "x[k] = v > 0.0f ? 1 : -1;"),
    ("no clamp", "if (clamp) { if", "if (0) { if"),
    ("penalty drops a check", "for (int32_t e = C->sym_ptr[k]; e < C->sym_ptr[k + 1]; ++e) S += s[C->chk_idx[e]];",
     "for (int32_t e = C->sym_ptr[k]; e + 1 < C->sym_ptr[k + 1]; ++e) S += s[C->chk_idx[e]];"),
    ("syndrome drops a symbol", "for (int32_t e = C->row_ptr[i]; e < C->row_ptr[i + 1]; ++e) prod *= x[C->col_idx[e]];",
     "for (int32_t e = C->row_ptr[i]; e + 1 < C->row_ptr[i + 1]; ++e) prod *= x[C->col_idx[e]];"),
    ("csc transposed", "C->chk_idx[fill[col_idx[e]]++] = i;", "C->chk_idx[fill[col_idx[e]]++] = col_idx[e] % m;"),
    ("sequential update", "if (flip) x[k] = (int8_t)-x[k];",
     "if (flip) { x[k] = (int8_t)-x[k]; for (int32_t e = C->sym_ptr[k]; e < C->sym_ptr[k + 1]; ++e) s[C->chk_idx[e]] = (int8_t)-s[C->chk_idx[e]]; }"),
    ("frame id offset", "J->frame_offset + (uint64_t)f,", "J->frame_offset + (uint64_t)f + 1,"),
    ("half rounding mode", "rint(fabs((double)x) / q) * q", "floor(fabs((double)x) / q) * q"),
    ("half quantum", "e >= -14 ? e - 10 : -24", "e >= -14 ? e - 11 : -24"),
    ("half overflow", "if (a >= 0x477FF000u)", "if (a >= 0x477FE000u)"),
    ("f16 metric drops a rounding", "const float e1 = oracle_round_half(xy + ws);", "const float e1 = xy + ws;"),
    ("f16 metric drops q rounding", "const float q16 = oracle_round_half(q);", "const float q16 = q;"),
    ("fix scale", "return (float)(ldexp(1.0, q_bits) / (2.0 * (double)y_max));",
     "return (float)(ldexp(1.0, q_bits) / (double)y_max);"),
    ("fix saturation", "X.fix_kmax = (1 << (P->q_bits - 1)) - 1;", "X.fix_kmax = (1 << (P->q_bits - 1));"),
    ("fix negative code", "return v >= 0.0f ? k : -k - 1;", "return v >= 0.0f ? k : -k;"),
    ("fix value", "return 2 * oracle_fix_code(v, R, kmax) + 1;", "return 2 * oracle_fix_code(v, R, kmax);"),
    ("fix weight", "X.fix_W = fix_value(P->w, X.fix_R, X.fix_kmax);", "X.fix_W = fix_value(P->w, X.fix_R, X.fix_kmax) + 2;"),
    ("single-bit tie to the higher index", "if (single && (best_k < 0 || E < best32)) { best_k = k; best32 = E; }\n                }\n            }",
     "if (single && (best_k < 0 || E <= best32)) { best_k = k; best32 = E; }\n                }\n            }"),
    ("single-bit flips every symbol", "            if (single) continue;\n", ""),
    ("fix metric sign", "const int32_t Eq = x[k] * yfix[k] + X->fix_W * S", "const int32_t Eq = x[k] * yfix[k] - X->fix_W * S"),
    ("uniform centre", "(int32_t)(2u * (r >> 8) + 1u) - (1 << 24)", "(int32_t)(2u * (r >> 8) + 1u) - (1 << 23)"),
    ("uniform bits", "const int32_t odd = (int32_t)(2u * (r >> 8) + 1u)", "const int32_t odd = (int32_t)(2u * (r >> 9) + 1u)"),
    ("uniform scale", "((double)P->eta * (double)sigma) * sqrt(3.0)", "((double)P->eta * (double)sigma) * sqrt(2.0)"),
    ("uniform bit ignored", "if (uniform) oracle_uniform4_f32(X->seed, frame_id, (uint32_t)t, (uint32_t)(k >> 2), z32);",
     "if (0) oracle_uniform4_f32(X->seed, frame_id, (uint32_t)t, (uint32_t)(k >> 2), z32);"),
    ("uniform output order", "for (int i = 0; i < 4; ++i) v[i] = oracle_uniform_f32(r[i]);",
     "for (int i = 0; i < 4; ++i) v[i] = oracle_uniform_f32(r[3 - i]);"),
    ("fixacc step count", "ldexp(1.0, q_bits + ORC_ACC_BITS)", "ldexp(1.0, q_bits + ORC_ACC_BITS + 1)"),
    ("fixacc held scale", "x[k] * yfix[k] * (1 << ORC_ACC_BITS)", "x[k] * yfix[k] * (1 << (ORC_ACC_BITS - 1))"),
    ("fixacc truncates", "return (int32_t)lrintf(a);", "return (int32_t)a;"),
    ("fixacc tie flips", "flip = Ea < X->thr_fix[u[k]];", "flip = Ea <= X->thr_fix[u[k]];"),
    ("fixacc weight from levels", "X.acc_W = oracle_fixacc_steps(P->w, X.acc_R);",
     "X.acc_W = X.fix_W * (1 << ORC_ACC_BITS);"),
    ("fixacc threshold from levels", ": X.precision == ORC_FIXACC ? oracle_fixacc_steps(thr32[u], X.acc_R) : 0;",
     ": X.precision == ORC_FIXACC ? fix_value(thr32[u], X.fix_R, X.fix_kmax) * (1 << ORC_ACC_BITS) : 0;"),
    ("fixacc drops the perturbation", "X->acc_W * S +\n                                       oracle_fixacc_steps(q, X->acc_R);",
     "X->acc_W * S;"),
    ("trace counts satisfied checks", "tr_u[t] = unsat;", "tr_u[t] = m - unsat;"),
    ("trace skips t = 0", "if (tr_u) {\n            tr_u[t]", "if (tr_u && t > 0) {\n            tr_u[t]"),
    ("trace uses raw samples", "? (double)yfix[k] * X->y_unit", "? ys64[k]"),
    ("trace unit", "llrint(ldexp((double)x[k] * yv, 32))", "llrint(ldexp((double)x[k] * yv, 31))"),
    ("trace level value", "X.y_unit = ldexp((double)P->y_max, -P->q_bits);", "X.y_unit = ldexp((double)P->y_max, 1 - P->q_bits);"),
]

RUNNER = r"""
import sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import oracle, oracle_pins
O = oracle.Oracle({lib!r})
for pin in oracle_pins.ALL_PINS:
    try:
        pin(O)
    except AssertionError as e:
        print("CAUGHT", pin.__name__, str(e)[:200])
        sys.exit(0)
print("NOT CAUGHT")
sys.exit(3)
"""


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new):
    src = open(oracle_pkg.SRC).read()
    assert src.count(old) == 1, f"mutation site for '{name}' must be unique"
    mutated = src.replace(old, new)
    path = tmp_path / "mutant.c"
    path.write_text(mutated)
    lib = str(tmp_path / "libmutant.so")
    oracle_pkg.compile_lib(str(path), lib)
    code = RUNNER.format(root=ROOT, tests=HERE, lib=lib)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode != 3, f"mutant '{name}' passed every pin:\n{r.stdout}\n{r.stderr}"
    # a crash or a caught assertion both count as detection
    assert "CAUGHT" in r.stdout or r.returncode != 0, r.stdout + r.stderr
