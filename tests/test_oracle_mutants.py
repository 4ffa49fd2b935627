"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in a temporary copy of oracle/gp_oracle.c,
builds it, and runs tests/test_oracle_pins.py against the copy: the pins
must fail.  Nothing here touches the real oracle or a GPU.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "gp_oracle.c")

MUTANTS = {
    "operand_order": ("double left = st[sp - 1], right = st[sp - 2];",
                      "double left = st[sp - 2], right = st[sp - 1];"),
    "fp32_operand_order": ("float left = st[sp - 1], right = st[sp - 2];",
                           "float left = st[sp - 2], right = st[sp - 1];"),
    "div_protect_value": ("case ORA_DIV: return fabs(b) < thr ? 1.0 : a / b;",
                          "case ORA_DIV: return fabs(b) < thr ? 0.0 : a / b;"),
    "threshold_inclusive": ("case ORA_DIV: return fabs(b) < thr ? 1.0 : a / b;",
                            "case ORA_DIV: return fabs(b) <= thr ? 1.0 : a / b;"),
    "sqrt_no_abs": ("case ORA_SQRT: return sqrt(fabs(a));", "case ORA_SQRT: return sqrt(a);"),
    "dropped_weight": ("se += wi * ora_loss(metric, v, (double)y[r]);",
                       "se += ora_loss(metric, v, (double)y[r]);"),
    "rmse_no_root": ("if (metric == ORA_RMSE) f = sqrt(f);", "if (0) f = sqrt(f);"),
    "logloss_label_swap": ("double c = (p >= 0.0) ? 1.0 - y : y;",
                           "double c = (p >= 0.0) ? y : 1.0 - y;"),
    "philox_9_rounds": ("for (int r = 0; r < 10; ++r) {", "for (int r = 0; r < 9; ++r) {"),
    "draw_word": ("(uint64_t)o[j & 3]", "(uint64_t)o[0]"),
    "tie_to_last": ("else better = adj < best_adj;", "else better = adj <= best_adj;"),
    "stack_bound_off_by_one": ("if (mx > ORA_MAX_STACK) return ORA_TOO_DEEP;",
                               "if (mx >= ORA_MAX_STACK) return ORA_TOO_DEEP;"),
    "dsub_sign": ("case ORA_SUB: du = 1.0; dv = -1.0; break;",
                  "case ORA_SUB: du = 1.0; dv = 1.0; break;"),
    "dmae_sign": ("case ORA_MAE: return sgn(p - y);", "case ORA_MAE: return sgn(y - p);"),
    "dcos_sign": ("case ORA_COS:  du = -sin(u); break;", "case ORA_COS:  du = sin(u); break;"),
    "adam_no_bias_correction": ("double mh = m[i] / b1t, vh = v[i] / b2t;",
                                "double mh = m[i], vh = v[i] / b2t;"),
    "pearson_p_not_centred": ("spp += wi * dp * dp;", "spp += wi * v * v;"),
    "pearson_signed": ("else f = fabs(spy / sqrt(spp * syy));", "else f = spy / sqrt(spp * syy);"),
    "ranks_without_tie_average": ("        double r = 0.5 * (double)(a + 1 + b + 1);  /* mean of positions a+1..b+1 */",
                                  "        double r = (double)(a + 1);"),
    "cube_as_square": ("    case ORA_CUBE: return a * a * a;", "    case ORA_CUBE: return a * a;"),
    "max_picks_smaller": ("     * operand when they compare equal */\n    case ORA_MAX: return (a > b || isnan(a)) ? a : b;",
                          "     * operand when they compare equal */\n    case ORA_MAX: return (a < b || isnan(a)) ? a : b;"),
    "dtanh_sign": ("                case ORA_TANH: du = 1.0 - val[j] * val[j]; break;",
                   "                case ORA_TANH: du = 1.0 + val[j] * val[j]; break;"),
    "hoist_from_anywhere": ("int k = si > 1 ? i + 1 + pick(&s, si - 1) : i;",
                            "int k = pick(&s, lp);"),
    "crossover_not_hoisted": ("        if (sj == 1) return 0; /* a terminal always fits a valid parent */",
                              "        return 0;"),
    "point_any_arity": ("                    const int *same = a == 1 ? f1 : f2;",
                        "                    const int *same = f2;"),
    "kind_thresholds_not_cumulative": ("        cum += probs[q];", "        cum = probs[q];"),
    "constant_half_range": ("        nd.c = (float)(w >> 8) * 0x1p-23f - 1.0f;",
                            "        nd.c = (float)(w >> 8) * 0x1p-24f - 1.0f;"),
    "grow_ignores_limit": ("        int terminal = d >= limit || pick(s, nf + 2) < 2;",
                           "        int terminal = d >= limit + 1 || pick(s, nf + 2) < 2;"),
    "bound_drops_mul_term": ("r.e = fabs(a.v) * b.e + fabs(b.v) * a.e + a.e * b.e;",
                             "r.e = fabs(a.v) * b.e + a.e * b.e;"),
    "bound_div_drops_b_term": (
        "        if (b.e < bv) r.e = (a.e + fabs(r.v) * b.e) / (bv - b.e);",
        "        if (b.e < bv) r.e = a.e / (bv - b.e);"),
    "bound_add_max_not_sum": ("        r.e = a.e + b.e;\n        return ve_round(r, 0.5);",
                              "        r.e = fmax(a.e, b.e);\n        return ve_round(r, 0.5);"),
    "bound_exp_no_growth": ("        r.e = fabs(r.v) * expm1(a.e);", "        r.e = a.e;"),
    "bound_sq_drops_linear": ("        r.e = 2.0 * av * a.e + a.e * a.e;", "        r.e = a.e * a.e;"),
    "parsimony_sign": ("adj = raw + pen;", "adj = raw - pen;"),
    "nan_counts_as_best": ("if (isnan(adj)) adj = INFINITY;", "if (isnan(adj)) adj = -INFINITY;"),
    "log_protect_value": ("case ORA_LOG:  return fabs(a) < thr ? 0.0 : log(fabs(a));",
                          "case ORA_LOG:  return fabs(a) < thr ? 1.0 : log(fabs(a));"),
    "inv_protect_value": ("case ORA_INV:  return fabs(a) < thr ? 0.0 : 1.0 / a;",
                          "case ORA_INV:  return fabs(a) < thr ? 1.0 : 1.0 / a;"),
    "mean_over_rows_not_weights": ("f = se / sw;", "f = se / (double)n_eval;"),
    "pearson_zero_variance_one": ("else if (spp == 0.0 || syy == 0.0) f = 0.0;",
                                  "else if (spp == 0.0 || syy == 0.0) f = 1.0;"),
    "draw_by_modulo": ("return (int64_t)(((uint64_t)o[j & 3] * (uint64_t)n_progs) >> 32);",
                       "return (int64_t)(o[j & 3] % (uint32_t)n_progs);"),
    "draw_counter_swapped": ("uint32_t ctr[4] = {(uint32_t)(j >> 2), (uint32_t)t, (uint32_t)offset,",
                             "uint32_t ctr[4] = {(uint32_t)t, (uint32_t)(j >> 2), (uint32_t)offset,"),
    "philox_key_schedule": ("k0 += W0; k1 += W1;", "k0 += W0; k1 += W0;"),
    "drmse_no_half": ("            scale = (f > 0.0) ? scale / (2.0 * f) : 0.0;\n        }\n"
                      "        for (int k = 0; k < ORA_MAX_CONSTS; ++k) {\n"
                      "            grad[p * ORA_MAX_CONSTS + k] = (k < nc) ? g[k] * scale : 0.0;\n"
                      "            /* sum of |per-row",
                      "            scale = (f > 0.0) ? scale / f : 0.0;\n        }\n"
                      "        for (int k = 0; k < ORA_MAX_CONSTS; ++k) {\n"
                      "            grad[p * ORA_MAX_CONSTS + k] = (k < nc) ? g[k] * scale : 0.0;\n"
                      "            /* sum of |per-row"),
    "feature_bound_off_by_one": (
        "        if (p[j].op == ORA_VAR && (p[j].feat < 0 || p[j].feat >= n_feat))",
        "        if (p[j].op == ORA_VAR && (p[j].feat < 0 || p[j].feat > n_feat))"),
    "adam_v_not_squared": ("        v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];",
                           "        v[i] = beta2 * v[i] + (1.0 - beta2) * fabs(g[i]);"),
    "rank_pearson_mean_unweighted": ("        sb += wi * b[i];", "        sb += b[i];"),
    "pearson_mean_unweighted": ("            swp += (w ? (double)w[row0 + i] : 1.0) * v;",
                                "            swp += v;"),
    "pearson_var_unweighted": ("                spp += wi * dp * dp;", "                spp += dp * dp;"),
    "dcosh_sign": ("                case ORA_COSH: du = sinh(u); break;",
                   "                case ORA_COSH: du = -sinh(u); break;"),
    "datan_no_square": ("                case ORA_ATAN: du = 1.0 / (1.0 + u * u); break;",
                        "                case ORA_ATAN: du = 1.0 / (1.0 + u); break;"),
    "sinh_as_cosh": ("    case ORA_SINH: return sinh(a);", "    case ORA_SINH: return cosh(a);"),
    "crossover_donor_is_parent": (
        "            int j = pick(&s, ld);\n"
        "            len = hoisted_splice(&s, par, lp, i, don, ld, j, child);",
        "            int j = pick(&s, lp);\n"
        "            len = hoisted_splice(&s, par, lp, i, par, lp, j, child);"),
    "point_replace_inverted": (
        "                if ((uint64_t)stream_next(&s) >= thr_replace) continue;",
        "                if ((uint64_t)stream_next(&s) < thr_replace) continue;"),
    "hoist_may_keep_root": ("            int k = si > 1 ? i + 1 + pick(&s, si - 1) : i;",
                            "            int k = si > 1 ? i + pick(&s, si) : i;"),
    "subtree_depth_plus_one": (
        "            int lt = grow_tree(&s, subtree_depth, funcs, nf, n_feat, tree);",
        "            int lt = grow_tree(&s, subtree_depth + 1, funcs, nf, n_feat, tree);"),
    "dlogloss_sign": ("                              : exp(p) / (1.0 + exp(p));\n        return s - y;",
                      "                              : exp(p) / (1.0 + exp(p));\n        return y - s;"),
    # the FP32 reverse mode (ora_const_grad32)
    "dcos32_sign": ("                case ORA_COS:  du = -sinf(u); break;",
                    "                case ORA_COS:  du = sinf(u); break;"),
    "dsqrt32_no_half": (
        "                case ORA_SQRT: du = (u == 0.0f) ? 0.0f : sgn32(u) / (2.0f * val[j]); break;",
        "                case ORA_SQRT: du = (u == 0.0f) ? 0.0f : sgn32(u) / val[j]; break;"),
    "dinv32_sign": (
        "                case ORA_INV:  du = (fabsf(u) < ORA_THR) ? 0.0f : -(val[j] * val[j]); break;",
        "                case ORA_INV:  du = (fabsf(u) < ORA_THR) ? 0.0f : (val[j] * val[j]); break;"),
    "ddiv32_right_sign": ("                    else { du = 1.0f / v; dv = -(val[j] / v); }",
                          "                    else { du = 1.0f / v; dv = (val[j] / v); }"),
    "dlogloss32_sign": (
        "        float s = (p >= 0.0f) ? 1.0f / (1.0f + expf(-p)) : expf(p) / (1.0f + expf(p));\n"
        "        return s - y;",
        "        float s = (p >= 0.0f) ? 1.0f / (1.0f + expf(-p)) : expf(p) / (1.0f + expf(p));\n"
        "        return y - s;"),
    "drmse32_no_half": (
        "            scale = (f > 0.0) ? scale / (2.0 * f) : 0.0;\n        }\n"
        "        for (int k = 0; k < ORA_MAX_CONSTS; ++k)\n"
        "            grad[p * ORA_MAX_CONSTS + k] = (k < nc) ? g[k] * scale : 0.0;",
        "            scale = (f > 0.0) ? scale / f : 0.0;\n        }\n"
        "        for (int k = 0; k < ORA_MAX_CONSTS; ++k)\n"
        "            grad[p * ORA_MAX_CONSTS + k] = (k < nc) ? g[k] * scale : 0.0;"),
    "dmae32_sign": ("    case ORA_MAE: return sgn32(p - y);", "    case ORA_MAE: return sgn32(y - p);"),
    "dabs32_one": ("                case ORA_ABS:  du = sgn32(u); break;",
                   "                case ORA_ABS:  du = 1.0f; break;"),
    "weight32_dropped_from_adjoint": ("            adj[0] = wi * dloss32(metric, pr, yi);",
                                      "            adj[0] = dloss32(metric, pr, yi);"),
    "dsin32_as_sin": ("                case ORA_SIN:  du = cosf(u); break;",
                      "                case ORA_SIN:  du = sinf(u); break;"),
}


def _run_mutant(name, tmp):
    old, new = MUTANTS[name]
    with open(SRC) as f:
        src = f.read()
    assert src.count(old) == 1, name
    d = os.path.join(tmp, name)
    os.makedirs(d, exist_ok=True)
    c = os.path.join(d, "m.c")
    so = os.path.join(d, "m.so")
    with open(c, "w") as f:
        f.write(src.replace(old, new))
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                    "-ffp-contract=off", c, "-o", so, "-lm"], check=True)
    # one OpenMP thread per mutant: the mutants already run side by side
    env = dict(os.environ, GP_ORACLE_SO=so, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_mutation.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return name, r.returncode


def test_pins_catch_planted_mistakes(tmp_path):
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        results = list(ex.map(lambda n: _run_mutant(n, str(tmp_path)), MUTANTS))
    survived = [n for n, rc in results if rc == 0]
    assert not survived, f"mutants not caught by the pins: {survived}"
