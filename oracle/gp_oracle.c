/*
 * gp_oracle.c -- plain, slow, obviously-correct CPU oracle for stack-based
 * genetic-programming fitness evaluation (Sathia, Ganesh, Nanditale,
 * "Accelerating Genetic Programming using GPUs", arXiv 2110.11226).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file: only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py use it.  It shares no code, header, table or
 * constant with the CUDA library; its op numbering and node layout are
 * written out here on their own and a test checks them against the
 * library's public header.
 *
 * Passages followed (section / equation of the paper):
 *   - Program = prefix (Polish) list of nodes, evaluated with a stack by a
 *     reverse scan of the list (Sec. III-A).
 *   - Functions have arity <= 2 (Sec. III); a stack of size m evaluates a
 *     tree of depth m-1 (Sec. III-C2, hoisted crossover), the stack size is
 *     20.
 *   - Fitness = weighted loss of the predictions against y, reduced per
 *     program (Sec. III-C3): MAE, MSE, RMSE, logistic loss; and the
 *     weighted Karl Pearson correlation coefficient of the predictions
 *     with y (Sec. III-C3 metric list).
 *   - Tournament selection: k Philox draws per tournament, best adjusted
 *     fitness wins, adjusted = raw + c * len (Sec. III-C1, Eqs. parsimony
 *     and fitness); Philox4x32-10 from Salmon et al. 2011 (Sec. III-B).
 *
 * Readings where the paper is silent:
 *   - first pop of a binary function is its LEFT operand;
 *   - protected operators with threshold 0.001f, compared as |x| < thr:
 *     div -> 1, inv -> 0, log -> 0, sqrt takes |x|; exp/sin/cos/tan plain;
 *   - weighted means normalised by sum(w); RMSE = sqrt(weighted MSE);
 *   - log-loss on sigmoid(p): c*|p| + log1p(exp(-|p|)), c = 1-y if p>=0
 *     else y, with the c*|p| term dropped when c == 0;
 *   - tournament draws with replacement, index = (u * n) >> 32, ties go to
 *     the earliest draw, NaN counts as the worst fitness;
 *   - Pearson fitness = |r_w(p, y)| with weighted means and (co)variances,
 *     greater is better, and 0 when either variance is 0;
 *   - Spearman fitness = the Pearson fitness of the average ranks;
 *   - the function set beyond the paper's benchmark set: sq, cube, cbrt,
 *     tanh, atan, sinh, cosh (unprotected) and max, min (NaN if either
 *     operand is NaN, the right operand when the two compare equal).
 *
 * Everything is FP64 unless a function says FP32 ("_f32" evaluates every
 * operation rounded to float with the C library's float functions; it is
 * the reference for bit-exact checks of the IEEE operators).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- node layout and op numbering (the library's input format) ---------- */
typedef struct {
    int16_t op;   /* opcode, see below                                  */
    int16_t feat; /* feature (column) index for a variable terminal     */
    float c;      /* value of a constant terminal                       */
} ora_node;

enum {
    ORA_CONST = 0, ORA_VAR = 1,
    ORA_ADD = 2, ORA_SUB = 3, ORA_MUL = 4, ORA_DIV = 5,
    ORA_SQRT = 6, ORA_LOG = 7, ORA_EXP = 8, ORA_SIN = 9, ORA_COS = 10,
    ORA_TAN = 11, ORA_ABS = 12, ORA_NEG = 13, ORA_INV = 14,
    ORA_SQ = 15, ORA_CUBE = 16, ORA_CBRT = 17, ORA_TANH = 18, ORA_ATAN = 19,
    ORA_SINH = 20, ORA_COSH = 21, ORA_MAX = 22, ORA_MIN = 23,
    ORA_NOPS = 24
};

enum { ORA_MAE = 0, ORA_MSE = 1, ORA_RMSE = 2, ORA_LOGLOSS = 3, ORA_PEARSON = 4,
       ORA_SPEARMAN = 5 };

#define ORA_MAX_STACK 20
#define ORA_MAX_LEN 255
#define ORA_MAX_CONSTS 16

/* status codes of ora_validate */
enum {
    ORA_OK = 0, ORA_BAD_LENGTH = 1, ORA_BAD_OP = 2, ORA_BAD_FEATURE = 3,
    ORA_UNDERFLOW = 4, ORA_LEFTOVER = 5, ORA_TOO_DEEP = 6
};

static const float ORA_THR = 0.001f;

static const char *const ora_names[ORA_NOPS] = {
    "const", "var", "add", "sub", "mul", "div", "sqrt", "log", "exp",
    "sin", "cos", "tan", "abs", "neg", "inv", "sq", "cube", "cbrt", "tanh",
    "atan", "sinh", "cosh", "max", "min"};

const char *ora_op_name(int op) {
    return (op >= 0 && op < ORA_NOPS) ? ora_names[op] : "";
}

int ora_op_arity(int op) {
    if (op == ORA_CONST || op == ORA_VAR) return 0;
    if ((op >= ORA_ADD && op <= ORA_DIV) || op == ORA_MAX || op == ORA_MIN) return 2;
    if (op >= ORA_SQRT && op <= ORA_COSH) return 1;
    return -1;
}

int ora_num_ops(void) { return ORA_NOPS; }

/* ---- validation: the reverse scan's stack high-water mark ------------- */
/* Returns a status code; *hw receives the largest stack height reached. */
int ora_validate(const ora_node *p, int len, int n_feat, int *hw) {
    int sp = 0, mx = 0;
    if (hw) *hw = 0;
    if (len < 1 || len > ORA_MAX_LEN) return ORA_BAD_LENGTH;
    for (int j = len - 1; j >= 0; --j) {
        int a = ora_op_arity(p[j].op);
        if (a < 0) return ORA_BAD_OP;
        if (p[j].op == ORA_VAR && (p[j].feat < 0 || p[j].feat >= n_feat))
            return ORA_BAD_FEATURE;
        if (a == 0) {
            sp += 1;
        } else {
            if (sp < a) return ORA_UNDERFLOW;
            sp -= a - 1;
        }
        if (sp > mx) mx = sp;
    }
    if (hw) *hw = mx;
    if (sp != 1) return ORA_LEFTOVER;
    if (mx > ORA_MAX_STACK) return ORA_TOO_DEEP;
    return ORA_OK;
}

/* ---- the function set, FP64 ------------------------------------------- */
static double fn1_64(int op, double a) {
    const double thr = (double)ORA_THR;
    switch (op) {
    case ORA_SQRT: return sqrt(fabs(a));
    case ORA_LOG:  return fabs(a) < thr ? 0.0 : log(fabs(a));
    case ORA_EXP:  return exp(a);
    case ORA_SIN:  return sin(a);
    case ORA_COS:  return cos(a);
    case ORA_TAN:  return tan(a);
    case ORA_ABS:  return fabs(a);
    case ORA_NEG:  return -a;
    case ORA_INV:  return fabs(a) < thr ? 0.0 : 1.0 / a;
    case ORA_SQ:   return a * a;
    case ORA_CUBE: return a * a * a;
    case ORA_CBRT: return cbrt(a);
    case ORA_TANH: return tanh(a);
    case ORA_ATAN: return atan(a);
    case ORA_SINH: return sinh(a);
    case ORA_COSH: return cosh(a);
    }
    return NAN;
}

/* a = left operand (first pop), b = right operand (second pop) */
static double fn2_64(int op, double a, double b) {
    const double thr = (double)ORA_THR;
    switch (op) {
    case ORA_ADD: return a + b;
    case ORA_SUB: return a - b;
    case ORA_MUL: return a * b;
    case ORA_DIV: return fabs(b) < thr ? 1.0 : a / b;
    /* the larger (smaller) operand; NaN if either is NaN; the right
     * operand when they compare equal */
    case ORA_MAX: return (a > b || isnan(a)) ? a : b;
    case ORA_MIN: return (a < b || isnan(a)) ? a : b;
    }
    return NAN;
}

/* ---- the function set, FP32 (every step rounded to float) ------------- */
static float fn1_32(int op, float a) {
    switch (op) {
    case ORA_SQRT: return sqrtf(fabsf(a));
    case ORA_LOG:  return fabsf(a) < ORA_THR ? 0.0f : logf(fabsf(a));
    case ORA_EXP:  return expf(a);
    case ORA_SIN:  return sinf(a);
    case ORA_COS:  return cosf(a);
    case ORA_TAN:  return tanf(a);
    case ORA_ABS:  return fabsf(a);
    case ORA_NEG:  return -a;
    case ORA_INV:  return fabsf(a) < ORA_THR ? 0.0f : 1.0f / a;
    case ORA_SQ:   return a * a;
    case ORA_CUBE: return (a * a) * a;
    case ORA_CBRT: return cbrtf(a);
    case ORA_TANH: return tanhf(a);
    case ORA_ATAN: return atanf(a);
    case ORA_SINH: return sinhf(a);
    case ORA_COSH: return coshf(a);
    }
    return NAN;
}

static float fn2_32(int op, float a, float b) {
    switch (op) {
    case ORA_ADD: return a + b;
    case ORA_SUB: return a - b;
    case ORA_MUL: return a * b;
    case ORA_DIV: return fabsf(b) < ORA_THR ? 1.0f : a / b;
    case ORA_MAX: return (a > b || isnan(a)) ? a : b;
    case ORA_MIN: return (a < b || isnan(a)) ? a : b;
    }
    return NAN;
}

/* ---- one program on one row: reverse scan of the prefix list ---------- */
/* X is column-major: X[f * ld + row].  Returns 0 or a status code; the
 * stack is as long as the program so any well-formed list evaluates. */
static int eval_row64(const ora_node *p, int len, const float *X, int64_t ld,
                      int64_t row, double *out) {
    double st[ORA_MAX_LEN + 1];
    int sp = 0;
    if (len < 1 || len > ORA_MAX_LEN) return ORA_BAD_LENGTH;
    for (int j = len - 1; j >= 0; --j) {
        int op = p[j].op, a = ora_op_arity(op);
        if (a < 0) return ORA_BAD_OP;
        if (op == ORA_CONST) {
            st[sp++] = (double)p[j].c;
        } else if (op == ORA_VAR) {
            st[sp++] = (double)X[(int64_t)p[j].feat * ld + row];
        } else if (a == 1) {
            if (sp < 1) return ORA_UNDERFLOW;
            st[sp - 1] = fn1_64(op, st[sp - 1]);
        } else {
            if (sp < 2) return ORA_UNDERFLOW;
            double left = st[sp - 1], right = st[sp - 2];
            sp -= 1;
            st[sp - 1] = fn2_64(op, left, right);
        }
    }
    if (sp != 1) return ORA_LEFTOVER;
    *out = st[0];
    return ORA_OK;
}

static int eval_row32(const ora_node *p, int len, const float *X, int64_t ld,
                      int64_t row, float *out) {
    float st[ORA_MAX_LEN + 1];
    int sp = 0;
    if (len < 1 || len > ORA_MAX_LEN) return ORA_BAD_LENGTH;
    for (int j = len - 1; j >= 0; --j) {
        int op = p[j].op, a = ora_op_arity(op);
        if (a < 0) return ORA_BAD_OP;
        if (op == ORA_CONST) {
            st[sp++] = p[j].c;
        } else if (op == ORA_VAR) {
            st[sp++] = X[(int64_t)p[j].feat * ld + row];
        } else if (a == 1) {
            if (sp < 1) return ORA_UNDERFLOW;
            st[sp - 1] = fn1_32(op, st[sp - 1]);
        } else {
            if (sp < 2) return ORA_UNDERFLOW;
            float left = st[sp - 1], right = st[sp - 2];
            sp -= 1;
            st[sp - 1] = fn2_32(op, left, right);
        }
    }
    if (sp != 1) return ORA_LEFTOVER;
    *out = st[0];
    return ORA_OK;
}

/* Predictions of every program on rows [row0, row0 + n_eval):
 * out[p * n_eval + i].  A malformed program gives NaN on every row; its
 * status goes to status[p] when status is not NULL. */
void ora_predict64(const ora_node *progs, const int32_t *offsets, int n_progs,
                   const float *X, int64_t ld, int64_t row0, int64_t n_eval,
                   double *out, int32_t *status, int n_threads) {
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic)
#endif
    for (int p = 0; p < n_progs; ++p) {
        const ora_node *prog = progs + offsets[p];
        int len = offsets[p + 1] - offsets[p];
        int st = ORA_OK;
        for (int64_t i = 0; i < n_eval; ++i) {
            double v = NAN;
            int s = eval_row64(prog, len, X, ld, row0 + i, &v);
            if (s) { st = s; v = NAN; }
            out[(int64_t)p * n_eval + i] = v;
        }
        if (status) status[p] = st;
    }
}

void ora_predict32(const ora_node *progs, const int32_t *offsets, int n_progs,
                   const float *X, int64_t ld, int64_t row0, int64_t n_eval,
                   float *out, int n_threads) {
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic)
#endif
    for (int p = 0; p < n_progs; ++p) {
        const ora_node *prog = progs + offsets[p];
        int len = offsets[p + 1] - offsets[p];
        for (int64_t i = 0; i < n_eval; ++i) {
            float v = NAN;
            if (eval_row32(prog, len, X, ld, row0 + i, &v)) v = NAN;
            out[(int64_t)p * n_eval + i] = v;
        }
    }
}

/* ---- running error bound of an FP32 evaluation ------------------------ *
 * Alongside the FP64 value v of every node this carries e, a first-order
 * bound on |v32 - v| for an evaluation that rounds each operation to
 * float and whose library functions err by at most ulps_fn units in the
 * last place.  Flags:
 *   1 = a protected operator's threshold test may decide differently in
 *       FP32 than in FP64 (the operand lies within e of the threshold);
 *   2 = an intermediate leaves the float range or becomes non-finite, or
 *       the bound itself is meaningless (tan near a pole, error larger
 *       than the operand of a division).
 * Textbook rules (Higham, "Accuracy and Stability of Numerical
 * Algorithms", 2nd ed., Ch. 2-3): |fl(x op y) - (x op y)| <= u |x op y|,
 * u = 2^-24, plus propagation of operand errors through first
 * derivatives. */
typedef struct { double v, e; int flags; } ora_ve;

static const double U32 = 5.9604644775390625e-08;   /* 2^-24 */
static const double ETA32 = 7.006492321624085e-46;  /* 2^-150: underflow */

static ora_ve ve_round(ora_ve r, double ulps) {
    /* rounding (or a library function's error) of the computed result,
     * |fl(x) - x| <= u|x| + eta with eta covering gradual underflow */
    double mag = fabs(r.v) + r.e;
    r.e += ulps * 2.0 * U32 * mag + ulps * 2.0 * ETA32;
    if (!isfinite(r.v) || fabs(r.v) > (double)FLT_MAX || !isfinite(r.e))
        r.flags |= 2;
    return r;
}

static ora_ve ve_fn2(int op, ora_ve a, ora_ve b);

static ora_ve ve_fn1(int op, ora_ve a, double ulps_fn) {
    const double thr = (double)ORA_THR;
    ora_ve r;
    r.flags = a.flags;
    r.v = fn1_64(op, a.v);
    double av = fabs(a.v);
    switch (op) {
    case ORA_ABS: case ORA_NEG:
        r.e = a.e;
        return r; /* exact operations */
    case ORA_SQRT:
        r.e = (av > 0.0) ? fmin(a.e / sqrt(av), sqrt(a.e)) : sqrt(a.e);
        return ve_round(r, 0.5);
    case ORA_LOG:
        if (fabs(av - thr) <= a.e) r.flags |= 1;
        if (av < thr) { r.e = 0.0; return r; }
        r.e = (a.e < av) ? -log1p(-a.e / av) : INFINITY;
        if (!(a.e < av)) r.flags |= 2;
        return ve_round(r, ulps_fn);
    case ORA_INV:
        if (fabs(av - thr) <= a.e) r.flags |= 1;
        if (av < thr) { r.e = 0.0; return r; }
        if (a.e < av) r.e = a.e / (av * (av - a.e));
        else { r.e = INFINITY; r.flags |= 2; }
        return ve_round(r, 0.5);
    case ORA_EXP:
        r.e = fabs(r.v) * expm1(a.e);
        return ve_round(r, ulps_fn);
    case ORA_SIN: case ORA_COS:
        r.e = fmin(a.e, 2.0);
        return ve_round(r, ulps_fn);
    case ORA_TAN: {
        double d = a.e * (1.0 + r.v * r.v);
        if (d > 0.1 * (1.0 + fabs(r.v))) { d = INFINITY; r.flags |= 2; }
        r.e = 2.0 * d; /* factor 2 covers the curvature over [a-e, a+e] */
        return ve_round(r, ulps_fn);
    }
    case ORA_SQ: /* one rounded product */
        r.e = 2.0 * av * a.e + a.e * a.e;
        return ve_round(r, 0.5);
    case ORA_CUBE: { /* two rounded products: (a*a)*a */
        ora_ve s = ve_fn2(ORA_MUL, a, a);
        return ve_fn2(ORA_MUL, s, a);
    }
    case ORA_CBRT: /* |cbrt(x)-cbrt(y)| <= 2^(2/3) |x-y|^(1/3); slope 1/(3 cbrt^2) */
        r.e = (fabs(r.v) > 0.0) ? fmin(a.e / (3.0 * r.v * r.v) * 2.0, 1.6 * cbrt(a.e))
                                : 1.6 * cbrt(a.e);
        return ve_round(r, ulps_fn);
    case ORA_TANH: /* slope <= 1 */
        r.e = fmin(a.e, 2.0);
        return ve_round(r, ulps_fn);
    case ORA_ATAN: { /* slope 1/(1+x^2) over [|a|-e, |a|+e] */
        double lo = fmax(0.0, av - a.e);
        r.e = a.e / (1.0 + lo * lo);
        return ve_round(r, ulps_fn);
    }
    case ORA_SINH: case ORA_COSH: /* slope <= cosh(|a|+e) */
        r.e = a.e * cosh(av + a.e);
        return ve_round(r, ulps_fn);
    }
    r.e = INFINITY;
    r.flags |= 2;
    return r;
}

static ora_ve ve_fn2(int op, ora_ve a, ora_ve b) {
    const double thr = (double)ORA_THR;
    ora_ve r;
    r.flags = a.flags | b.flags;
    r.v = fn2_64(op, a.v, b.v);
    switch (op) {
    case ORA_ADD: case ORA_SUB:
        r.e = a.e + b.e;
        return ve_round(r, 0.5);
    case ORA_MUL:
        r.e = fabs(a.v) * b.e + fabs(b.v) * a.e + a.e * b.e;
        return ve_round(r, 0.5);
    case ORA_DIV: {
        double bv = fabs(b.v);
        if (fabs(bv - thr) <= b.e) r.flags |= 1;
        if (bv < thr) { r.e = 0.0; return r; }
        if (b.e < bv) r.e = (a.e + fabs(r.v) * b.e) / (bv - b.e);
        else { r.e = INFINITY; r.flags |= 2; }
        return ve_round(r, 0.5);
    }
    case ORA_MAX: case ORA_MIN: /* 1-Lipschitz in each operand, exact */
        r.e = fmax(a.e, b.e);
        if (!isfinite(r.v)) r.flags |= 2;
        return r;
    }
    r.e = INFINITY;
    r.flags |= 2;
    return r;
}

static int eval_row_bound(const ora_node *p, int len, const float *X,
                          int64_t ld, int64_t row, double ulps_fn,
                          ora_ve *out) {
    ora_ve st[ORA_MAX_LEN + 1];
    int sp = 0;
    if (len < 1 || len > ORA_MAX_LEN) return ORA_BAD_LENGTH;
    for (int j = len - 1; j >= 0; --j) {
        int op = p[j].op, a = ora_op_arity(op);
        if (a < 0) return ORA_BAD_OP;
        if (op == ORA_CONST || op == ORA_VAR) {
            ora_ve t;
            t.v = (op == ORA_CONST) ? (double)p[j].c
                                    : (double)X[(int64_t)p[j].feat * ld + row];
            t.e = 0.0; /* inputs are floats: exact in both precisions */
            t.flags = isfinite(t.v) ? 0 : 2;
            st[sp++] = t;
        } else if (a == 1) {
            if (sp < 1) return ORA_UNDERFLOW;
            st[sp - 1] = ve_fn1(op, st[sp - 1], ulps_fn);
        } else {
            if (sp < 2) return ORA_UNDERFLOW;
            ora_ve left = st[sp - 1], right = st[sp - 2];
            sp -= 1;
            st[sp - 1] = ve_fn2(op, left, right);
        }
    }
    if (sp != 1) return ORA_LEFTOVER;
    *out = st[0];
    return ORA_OK;
}

void ora_predict_bound(const ora_node *progs, const int32_t *offsets,
                       int n_progs, const float *X, int64_t ld, int64_t row0,
                       int64_t n_eval, double ulps_fn, double *out_v,
                       double *out_e, uint8_t *out_flags, int n_threads) {
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic)
#endif
    for (int p = 0; p < n_progs; ++p) {
        const ora_node *prog = progs + offsets[p];
        int len = offsets[p + 1] - offsets[p];
        for (int64_t i = 0; i < n_eval; ++i) {
            ora_ve r;
            int64_t k = (int64_t)p * n_eval + i;
            if (eval_row_bound(prog, len, X, ld, row0 + i, ulps_fn, &r)) {
                r.v = NAN; r.e = INFINITY; r.flags = 2;
            }
            out_v[k] = r.v;
            out_e[k] = r.e;
            out_flags[k] = (uint8_t)r.flags;
        }
    }
}

/* ---- fitness ------------------------------------------------------------ */
/* Per-row loss of prediction p against target y (Sec. III-C3 metric list;
 * the formulas are the weighted-mean readings stated in the header). */
double ora_loss(int metric, double p, double y) {
    switch (metric) {
    case ORA_MAE: return fabs(p - y);
    case ORA_MSE: case ORA_RMSE: return (p - y) * (p - y);
    case ORA_LOGLOSS: {
        double ap = fabs(p);
        double c = (p >= 0.0) ? 1.0 - y : y;
        double lin = (c == 0.0) ? 0.0 : c * ap;
        return lin + log1p(exp(-ap));
    }
    }
    return NAN;
}

/* Fitness of every program over rows [row0, row0 + n_eval):
 *   MAE/MSE/logloss = sum_i w_i l_i / sum_i w_i, RMSE = sqrt(MSE).
 * w == NULL means all weights 1.  Returns 0, or -1 for a bad metric or a
 * zero total weight.  A malformed program gets NaN and status[p] != 0. */
static int pearson_fitness(const ora_node *progs, const int32_t *offsets, int n_progs,
                           const float *X, int64_t ld, const float *y, const float *w,
                           int64_t row0, int64_t n_eval, double sw, double *out_fit,
                           int32_t *status, int n_threads);
static int spearman_fitness(const ora_node *progs, const int32_t *offsets, int n_progs,
                            const float *X, int64_t ld, const float *y, const float *w,
                            int64_t row0, int64_t n_eval, double *out_fit, int32_t *status,
                            int n_threads);

int ora_fitness(const ora_node *progs, const int32_t *offsets, int n_progs,
                const float *X, int64_t ld, const float *y, const float *w,
                int metric, int64_t row0, int64_t n_eval, double *out_fit,
                int32_t *status, int n_threads) {
    if (metric < ORA_MAE || metric > ORA_SPEARMAN) return -1;
    double sw = 0.0;
    for (int64_t i = 0; i < n_eval; ++i) sw += w ? (double)w[row0 + i] : 1.0;
    if (!(sw != 0.0)) return -1;
    if (metric == ORA_PEARSON)
        return pearson_fitness(progs, offsets, n_progs, X, ld, y, w, row0, n_eval, sw, out_fit,
                               status, n_threads);
    if (metric == ORA_SPEARMAN)
        return spearman_fitness(progs, offsets, n_progs, X, ld, y, w, row0, n_eval, out_fit,
                                status, n_threads);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic)
#endif
    for (int p = 0; p < n_progs; ++p) {
        const ora_node *prog = progs + offsets[p];
        int len = offsets[p + 1] - offsets[p];
        double se = 0.0;
        int st = ORA_OK;
        for (int64_t i = 0; i < n_eval && st == ORA_OK; ++i) {
            double v;
            int64_t r = row0 + i;
            st = eval_row64(prog, len, X, ld, r, &v);
            if (st) break;
            double wi = w ? (double)w[r] : 1.0;
            se += wi * ora_loss(metric, v, (double)y[r]);
        }
        double f = NAN;
        if (st == ORA_OK) {
            f = se / sw;
            if (metric == ORA_RMSE) f = sqrt(f);
        }
        out_fit[p] = f;
        if (status) status[p] = st;
    }
    return 0;
}

/* Weighted Pearson correlation, by its definition with two passes over
 * the rows (Sec. III-C3 names the coefficient; the weighting follows the
 * other metrics):
 *   pbar = sum w p / sum w,  ybar = sum w y / sum w,
 *   r = sum w (p-pbar)(y-ybar) / sqrt(sum w (p-pbar)^2 * sum w (y-ybar)^2),
 * fitness = |r|, and 0 when either sum of squares is 0.  Non-finite
 * predictions give NaN. */
static int pearson_fitness(const ora_node *progs, const int32_t *offsets, int n_progs,
                           const float *X, int64_t ld, const float *y, const float *w,
                           int64_t row0, int64_t n_eval, double sw, double *out_fit,
                           int32_t *status, int n_threads) {
    double swy = 0.0;
    for (int64_t i = 0; i < n_eval; ++i)
        swy += (w ? (double)w[row0 + i] : 1.0) * (double)y[row0 + i];
    const double ybar = swy / sw;
    double syy = 0.0;
    for (int64_t i = 0; i < n_eval; ++i) {
        const double dy = (double)y[row0 + i] - ybar;
        syy += (w ? (double)w[row0 + i] : 1.0) * dy * dy;
    }
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic)
#endif
    for (int p = 0; p < n_progs; ++p) {
        const ora_node *prog = progs + offsets[p];
        int len = offsets[p + 1] - offsets[p];
        int st = ORA_OK;
        double swp = 0.0;
        for (int64_t i = 0; i < n_eval && st == ORA_OK; ++i) {
            double v;
            st = eval_row64(prog, len, X, ld, row0 + i, &v);
            if (st) break;
            swp += (w ? (double)w[row0 + i] : 1.0) * v;
        }
        double f = NAN;
        if (st == ORA_OK) {
            const double pbar = swp / sw;
            double spp = 0.0, spy = 0.0;
            for (int64_t i = 0; i < n_eval; ++i) {
                double v;
                eval_row64(prog, len, X, ld, row0 + i, &v);
                const double wi = w ? (double)w[row0 + i] : 1.0;
                const double dp = v - pbar;
                spp += wi * dp * dp;
                spy += wi * dp * ((double)y[row0 + i] - ybar);
            }
            if (isnan(spp) || isnan(spy) || isinf(spp) || isinf(spy)) f = NAN;
            else if (spp == 0.0 || syy == 0.0) f = 0.0;
            else f = fabs(spy / sqrt(spp * syy));
        }
        out_fit[p] = f;
        if (status) status[p] = st;
    }
    return 0;
}

/* Spearman's rank correlation (Sec. III-C3: the ranks of the values, then
 * Karl Pearson's coefficient of the ranks): rank = 1-based position in
 * ascending order, tied values sharing the mean of their positions; the
 * weighted Pearson coefficient of the two rank vectors, as a fitness |r|
 * (0 when either variance is 0, NaN when a value is NaN). */
static const double *g_sort_keys;
static int cmp_by_key(const void *a, const void *b) {
    double x = g_sort_keys[*(const int64_t *)a], y = g_sort_keys[*(const int64_t *)b];
    if (x < y) return -1;
    if (x > y) return 1;
    int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
    return (i > j) - (i < j);
}

/* average ranks of v[0..n) into rank[]; returns -1 if a value is NaN */
int ora_average_ranks(const double *v, int64_t n, double *rank) {
    for (int64_t i = 0; i < n; ++i)
        if (isnan(v[i])) return -1;
    int64_t *idx = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!idx) return -2;
    for (int64_t i = 0; i < n; ++i) idx[i] = i;
#ifdef _OPENMP
#pragma omp critical(ora_sort)
#endif
    {
        g_sort_keys = v;
        qsort(idx, (size_t)n, sizeof(int64_t), cmp_by_key);
    }
    for (int64_t a = 0; a < n;) {
        int64_t b = a;
        while (b + 1 < n && v[idx[b + 1]] == v[idx[a]]) ++b;
        double r = 0.5 * (double)(a + 1 + b + 1);  /* mean of positions a+1..b+1 */
        for (int64_t m = a; m <= b; ++m) rank[idx[m]] = r;
        a = b + 1;
    }
    free(idx);
    return 0;
}

/* |weighted Pearson| of two vectors by its two-pass definition */
double ora_weighted_abs_pearson(const double *a, const double *b, const float *w, int64_t n) {
    double sw = 0.0, sa = 0.0, sb = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double wi = w ? (double)w[i] : 1.0;
        sw += wi;
        sa += wi * a[i];
        sb += wi * b[i];
    }
    double ma = sa / sw, mb = sb / sw, saa = 0.0, sbb = 0.0, sab = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double wi = w ? (double)w[i] : 1.0;
        saa += wi * (a[i] - ma) * (a[i] - ma);
        sbb += wi * (b[i] - mb) * (b[i] - mb);
        sab += wi * (a[i] - ma) * (b[i] - mb);
    }
    if (isnan(saa) || isnan(sab) || isinf(saa) || isinf(sab)) return NAN;
    if (saa == 0.0 || sbb == 0.0) return 0.0;
    return fabs(sab / sqrt(saa * sbb));
}

/* Spearman fitness of given predictions p[0..n) against y (weights w) */
double ora_spearman_of(const double *p, const float *y, const float *w, int64_t n) {
    double *rp = (double *)malloc((size_t)n * sizeof(double));
    double *ry = (double *)malloc((size_t)n * sizeof(double));
    double *yd = (double *)malloc((size_t)n * sizeof(double));
    double f = NAN;
    if (rp && ry && yd) {
        for (int64_t i = 0; i < n; ++i) yd[i] = (double)y[i];
        if (ora_average_ranks(p, n, rp) == 0 && ora_average_ranks(yd, n, ry) == 0)
            f = ora_weighted_abs_pearson(rp, ry, w, n);
    }
    free(rp);
    free(ry);
    free(yd);
    return f;
}

static int spearman_fitness(const ora_node *progs, const int32_t *offsets, int n_progs,
                            const float *X, int64_t ld, const float *y, const float *w,
                            int64_t row0, int64_t n_eval, double *out_fit, int32_t *status,
                            int n_threads) {
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic)
#endif
    for (int p = 0; p < n_progs; ++p) {
        const ora_node *prog = progs + offsets[p];
        int len = offsets[p + 1] - offsets[p];
        double *v = (double *)malloc((size_t)n_eval * sizeof(double));
        int st = v ? ORA_OK : ORA_BAD_LENGTH;
        for (int64_t i = 0; i < n_eval && st == ORA_OK; ++i)
            st = eval_row64(prog, len, X, ld, row0 + i, &v[i]);
        out_fit[p] = st == ORA_OK ? ora_spearman_of(v, y + row0, w ? w + row0 : NULL, n_eval) : NAN;
        if (status) status[p] = st;
        free(v);
    }
    return 0;
}

/* ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ---------------- *
 * Round: with the 32x32->64 products of counter words 0 and 2 by the two
 * multipliers, the new counter is (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2),
 * hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)); the key advances by the two Weyl
 * constants between rounds; ten rounds. */
void ora_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Draw j of tournament t: counter (j/4, t, offset lo, offset hi), key
 * (seed lo, seed hi), output word j%4, index = (u * n_progs) >> 32. */
int64_t ora_tournament_draw(uint64_t seed, uint64_t offset, int64_t t, int j,
                            int n_progs) {
    uint32_t ctr[4] = {(uint32_t)(j >> 2), (uint32_t)t, (uint32_t)offset,
                       (uint32_t)(offset >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    ora_philox4x32_10(ctr, key, o);
    return (int64_t)(((uint64_t)o[j & 3] * (uint64_t)n_progs) >> 32);
}

/* Tournament selection (Sec. III-C1).  adjusted = raw + c*len when smaller
 * is better (Eqs. parsimony, fitness), raw - c*len when greater is better.
 * The winner is the draw with the strictly best adjusted fitness; the
 * first such draw wins ties; NaN is the worst value.  lengths may be NULL
 * (no penalty). */
int ora_tournament(const float *fitness, const int32_t *lengths, int n_progs,
                   int64_t n_tourn, int k, float parsimony,
                   int greater_is_better, uint64_t seed, uint64_t offset,
                   int32_t *out_idx) {
    if (n_progs < 1 || k < 1 || n_tourn < 0) return -1;
    for (int64_t t = 0; t < n_tourn; ++t) {
        int best = -1;
        double best_adj = 0.0;
        for (int j = 0; j < k; ++j) {
            int i = (int)ora_tournament_draw(seed, offset, t, j, n_progs);
            double pen = lengths ? (double)parsimony * (double)lengths[i] : 0.0;
            double raw = (double)fitness[i];
            double adj;
            if (greater_is_better) {
                adj = raw - pen;
                if (isnan(adj)) adj = -INFINITY;
            } else {
                adj = raw + pen;
                if (isnan(adj)) adj = INFINITY;
            }
            int better;
            if (best < 0) better = 1;
            else if (greater_is_better) better = adj > best_adj;
            else better = adj < best_adj;
            if (better) { best = i; best_adj = adj; }
        }
        out_idx[t] = best;
    }
    return 0;
}

/* ---- reverse mode: gradient of fitness w.r.t. the constants ----------- *
 * A tape of node values from the reverse scan, then adjoints pushed from
 * the root down in prefix order; constant k (k-th CONST node in prefix
 * order) collects the adjoint of its node.  Derivative of a protected
 * operator is 0 on its protected branch. */
static double sgn(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0); }

static double dloss(int metric, double p, double y) {
    switch (metric) {
    case ORA_MAE: return sgn(p - y);
    case ORA_MSE: case ORA_RMSE: return 2.0 * (p - y);
    case ORA_LOGLOSS: {
        double s = (p >= 0.0) ? 1.0 / (1.0 + exp(-p))
                              : exp(p) / (1.0 + exp(p));
        return s - y;
    }
    }
    return NAN;
}

int ora_count_consts(const ora_node *p, int len) {
    int n = 0;
    for (int j = 0; j < len; ++j) n += (p[j].op == ORA_CONST);
    return n;
}

/* grad[p * 16 + k] = d fitness_p / d c_k, fit[p] = fitness_p, gabs (may be
 * NULL) = the same sum over rows taken of absolute values.  Returns 0,
 * -1 (bad metric / zero weight) or -2 (a program with more than 16
 * constants; its row of grad is NaN). */
int ora_const_grad(const ora_node *progs, const int32_t *offsets,
                   int n_progs, const float *X, int64_t ld, const float *y,
                   const float *w, int metric, int64_t row0, int64_t n_eval,
                   double *grad, double *fit, double *gabs, int n_threads) {
    if (metric < ORA_MAE || metric > ORA_LOGLOSS) return -1;
    double sw = 0.0;
    for (int64_t i = 0; i < n_eval; ++i) sw += w ? (double)w[row0 + i] : 1.0;
    if (!(sw != 0.0)) return -1;
    int rc = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic) reduction(min : rc)
#endif
    for (int p = 0; p < n_progs; ++p) {
        const ora_node *prog = progs + offsets[p];
        int len = offsets[p + 1] - offsets[p];
        double g[ORA_MAX_CONSTS], ga[ORA_MAX_CONSTS];
        int kslot[ORA_MAX_LEN];
        for (int k = 0; k < ORA_MAX_CONSTS; ++k) g[k] = ga[k] = 0.0;
        int nc = 0, bad = 0;
        if (len < 1 || len > ORA_MAX_LEN) bad = 1;
        for (int j = 0; j < len && !bad; ++j) {
            kslot[j] = -1;
            if (prog[j].op == ORA_CONST) {
                if (nc >= ORA_MAX_CONSTS) { bad = 2; break; }
                kslot[j] = nc++;
            }
        }
        double se = 0.0;
        for (int64_t i = 0; i < n_eval && !bad; ++i) {
            int64_t r = row0 + i;
            double val[ORA_MAX_LEN], adj[ORA_MAX_LEN];
            int left[ORA_MAX_LEN], right[ORA_MAX_LEN];
            int pos[ORA_MAX_LEN + 1], sp = 0;
            /* forward: reverse scan; the stack holds node positions */
            for (int j = len - 1; j >= 0 && !bad; --j) {
                int op = prog[j].op, a = ora_op_arity(op);
                left[j] = right[j] = -1;
                if (a < 0) { bad = 1; break; }
                if (op == ORA_CONST) val[j] = (double)prog[j].c;
                else if (op == ORA_VAR)
                    val[j] = (double)X[(int64_t)prog[j].feat * ld + r];
                else if (a == 1) {
                    if (sp < 1) { bad = 1; break; }
                    left[j] = pos[--sp];
                    val[j] = fn1_64(op, val[left[j]]);
                } else {
                    if (sp < 2) { bad = 1; break; }
                    left[j] = pos[--sp];
                    right[j] = pos[--sp];
                    val[j] = fn2_64(op, val[left[j]], val[right[j]]);
                }
                pos[sp++] = j;
            }
            if (bad || sp != 1) { bad = 1; break; }
            double pr = val[0], yi = (double)y[r];
            double wi = w ? (double)w[r] : 1.0;
            se += wi * ora_loss(metric, pr, yi);
            /* backward: prefix order, parents before children */
            for (int j = 0; j < len; ++j) adj[j] = 0.0;
            adj[0] = wi * dloss(metric, pr, yi);
            const double thr = (double)ORA_THR;
            for (int j = 0; j < len; ++j) {
                int op = prog[j].op;
                double aj = adj[j];
                if (op == ORA_CONST) {
                    g[kslot[j]] += aj;
                    ga[kslot[j]] += fabs(aj);
                    continue;
                }
                if (op == ORA_VAR) continue;
                double u = val[left[j]];
                double du = 0.0, dv = 0.0;
                switch (op) {
                case ORA_ADD: du = 1.0; dv = 1.0; break;
                case ORA_SUB: du = 1.0; dv = -1.0; break;
                case ORA_MUL: du = val[right[j]]; dv = u; break;
                case ORA_DIV: {
                    double v = val[right[j]];
                    if (fabs(v) < thr) { du = 0.0; dv = 0.0; }
                    else { du = 1.0 / v; dv = -u / (v * v); }
                    break;
                }
                case ORA_SQRT: du = (u == 0.0) ? 0.0 : sgn(u) / (2.0 * sqrt(fabs(u))); break;
                case ORA_LOG:  du = (fabs(u) < thr) ? 0.0 : 1.0 / u; break;
                case ORA_EXP:  du = val[j]; break;
                case ORA_SIN:  du = cos(u); break;
                case ORA_COS:  du = -sin(u); break;
                case ORA_TAN:  du = 1.0 + val[j] * val[j]; break;
                case ORA_ABS:  du = sgn(u); break;
                case ORA_NEG:  du = -1.0; break;
                case ORA_INV:  du = (fabs(u) < thr) ? 0.0 : -1.0 / (u * u); break;
                case ORA_SQ:   du = 2.0 * u; break;
                case ORA_CUBE: du = 3.0 * u * u; break;
                case ORA_CBRT: du = (u == 0.0) ? 0.0 : 1.0 / (3.0 * val[j] * val[j]); break;
                case ORA_TANH: du = 1.0 - val[j] * val[j]; break;
                case ORA_ATAN: du = 1.0 / (1.0 + u * u); break;
                case ORA_SINH: du = cosh(u); break;
                case ORA_COSH: du = sinh(u); break;
                case ORA_MAX: {
                    int takes_left = u > val[right[j]] || isnan(u);
                    du = takes_left ? 1.0 : 0.0;
                    dv = 1.0 - du;
                    break;
                }
                case ORA_MIN: {
                    int takes_left = u < val[right[j]] || isnan(u);
                    du = takes_left ? 1.0 : 0.0;
                    dv = 1.0 - du;
                    break;
                }
                }
                adj[left[j]] = aj * du;
                if (right[j] >= 0) adj[right[j]] = aj * dv;
            }
        }
        if (bad) {
            for (int k = 0; k < ORA_MAX_CONSTS; ++k) {
                grad[p * ORA_MAX_CONSTS + k] = NAN;
                if (gabs) gabs[p * ORA_MAX_CONSTS + k] = NAN;
            }
            if (fit) fit[p] = NAN;
            if (bad == 2) rc = -2;
            continue;
        }
        double f = se / sw, scale = 1.0 / sw;
        if (metric == ORA_RMSE) {
            f = sqrt(f);
            scale = (f > 0.0) ? scale / (2.0 * f) : 0.0;
        }
        for (int k = 0; k < ORA_MAX_CONSTS; ++k) {
            grad[p * ORA_MAX_CONSTS + k] = (k < nc) ? g[k] * scale : 0.0;
            /* sum of |per-row contributions|: the scale of the gradient's
             * cancellation, used to state gradient tolerances */
            if (gabs) gabs[p * ORA_MAX_CONSTS + k] = (k < nc) ? ga[k] * fabs(scale) : 0.0;
        }
        if (fit) fit[p] = f;
    }
    return rc;
}

/* The same reverse mode with every per-row operation in FP32 (C library
 * float functions, derivatives formed in float) and only the sums over
 * rows in FP64.  Its distance from ora_const_grad measures how much FP32
 * rounding alone moves each gradient (the gradient's conditioning); it is
 * the reference the GPU's FP32 adjoint is held to where that distance is
 * large.  Same arguments and return values as ora_const_grad. */
static float sgn32(float x) { return x > 0.0f ? 1.0f : (x < 0.0f ? -1.0f : 0.0f); }

static float loss32(int metric, float p, float y) {
    switch (metric) {
    case ORA_MAE: return fabsf(p - y);
    case ORA_MSE: case ORA_RMSE: return (p - y) * (p - y);
    case ORA_LOGLOSS: {
        float ap = fabsf(p);
        float c = (p >= 0.0f) ? 1.0f - y : y;
        float lin = (c == 0.0f) ? 0.0f : c * ap;
        return lin + log1pf(expf(-ap));
    }
    }
    return NAN;
}

static float dloss32(int metric, float p, float y) {
    switch (metric) {
    case ORA_MAE: return sgn32(p - y);
    case ORA_MSE: case ORA_RMSE: return 2.0f * (p - y);
    case ORA_LOGLOSS: {
        float s = (p >= 0.0f) ? 1.0f / (1.0f + expf(-p)) : expf(p) / (1.0f + expf(p));
        return s - y;
    }
    }
    return NAN;
}

int ora_const_grad32(const ora_node *progs, const int32_t *offsets,
                     int n_progs, const float *X, int64_t ld, const float *y,
                     const float *w, int metric, int64_t row0, int64_t n_eval,
                     double *grad, double *fit, int n_threads) {
    if (metric < ORA_MAE || metric > ORA_LOGLOSS) return -1;
    double sw = 0.0;
    for (int64_t i = 0; i < n_eval; ++i) sw += w ? (double)w[row0 + i] : 1.0;
    if (!(sw != 0.0)) return -1;
    int rc = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic) reduction(min : rc)
#endif
    for (int p = 0; p < n_progs; ++p) {
        const ora_node *prog = progs + offsets[p];
        int len = offsets[p + 1] - offsets[p];
        double g[ORA_MAX_CONSTS];
        int kslot[ORA_MAX_LEN];
        for (int k = 0; k < ORA_MAX_CONSTS; ++k) g[k] = 0.0;
        int nc = 0, bad = 0;
        if (len < 1 || len > ORA_MAX_LEN) bad = 1;
        for (int j = 0; j < len && !bad; ++j) {
            kslot[j] = -1;
            if (prog[j].op == ORA_CONST) {
                if (nc >= ORA_MAX_CONSTS) { bad = 2; break; }
                kslot[j] = nc++;
            }
        }
        double se = 0.0;
        for (int64_t i = 0; i < n_eval && !bad; ++i) {
            int64_t r = row0 + i;
            float val[ORA_MAX_LEN], adj[ORA_MAX_LEN];
            int left[ORA_MAX_LEN], right[ORA_MAX_LEN];
            int pos[ORA_MAX_LEN + 1], sp = 0;
            for (int j = len - 1; j >= 0 && !bad; --j) {
                int op = prog[j].op, a = ora_op_arity(op);
                left[j] = right[j] = -1;
                if (a < 0) { bad = 1; break; }
                if (op == ORA_CONST) val[j] = prog[j].c;
                else if (op == ORA_VAR) val[j] = X[(int64_t)prog[j].feat * ld + r];
                else if (a == 1) {
                    if (sp < 1) { bad = 1; break; }
                    left[j] = pos[--sp];
                    val[j] = fn1_32(op, val[left[j]]);
                } else {
                    if (sp < 2) { bad = 1; break; }
                    left[j] = pos[--sp];
                    right[j] = pos[--sp];
                    val[j] = fn2_32(op, val[left[j]], val[right[j]]);
                }
                pos[sp++] = j;
            }
            if (bad || sp != 1) { bad = 1; break; }
            float pr = val[0], yi = y[r];
            float wi = w ? w[r] : 1.0f;
            se += (double)(wi * loss32(metric, pr, yi));
            for (int j = 0; j < len; ++j) adj[j] = 0.0f;
            adj[0] = wi * dloss32(metric, pr, yi);
            for (int j = 0; j < len; ++j) {
                int op = prog[j].op;
                float aj = adj[j];
                if (op == ORA_CONST) { g[kslot[j]] += (double)aj; continue; }
                if (op == ORA_VAR) continue;
                float u = val[left[j]];
                float du = 0.0f, dv = 0.0f;
                switch (op) {
                case ORA_ADD: du = 1.0f; dv = 1.0f; break;
                case ORA_SUB: du = 1.0f; dv = -1.0f; break;
                case ORA_MUL: du = val[right[j]]; dv = u; break;
                case ORA_DIV: {
                    float v = val[right[j]];
                    if (fabsf(v) < ORA_THR) { du = 0.0f; dv = 0.0f; }
                    else { du = 1.0f / v; dv = -(val[j] / v); }
                    break;
                }
                case ORA_SQRT: du = (u == 0.0f) ? 0.0f : sgn32(u) / (2.0f * val[j]); break;
                case ORA_LOG:  du = (fabsf(u) < ORA_THR) ? 0.0f : 1.0f / u; break;
                case ORA_EXP:  du = val[j]; break;
                case ORA_SIN:  du = cosf(u); break;
                case ORA_COS:  du = -sinf(u); break;
                case ORA_TAN:  du = 1.0f + val[j] * val[j]; break;
                case ORA_ABS:  du = sgn32(u); break;
                case ORA_NEG:  du = -1.0f; break;
                case ORA_INV:  du = (fabsf(u) < ORA_THR) ? 0.0f : -(val[j] * val[j]); break;
                case ORA_SQ:   du = 2.0f * u; break;
                case ORA_CUBE: du = 3.0f * (u * u); break;
                case ORA_CBRT: du = (u == 0.0f) ? 0.0f : 1.0f / (3.0f * (val[j] * val[j])); break;
                case ORA_TANH: du = 1.0f - val[j] * val[j]; break;
                case ORA_ATAN: du = 1.0f / (1.0f + u * u); break;
                case ORA_SINH: du = coshf(u); break;
                case ORA_COSH: du = sinhf(u); break;
                case ORA_MAX: {
                    int takes_left = u > val[right[j]] || isnan(u);
                    du = takes_left ? 1.0f : 0.0f;
                    dv = 1.0f - du;
                    break;
                }
                case ORA_MIN: {
                    int takes_left = u < val[right[j]] || isnan(u);
                    du = takes_left ? 1.0f : 0.0f;
                    dv = 1.0f - du;
                    break;
                }
                }
                adj[left[j]] = aj * du;
                if (right[j] >= 0) adj[right[j]] = aj * dv;
            }
        }
        if (bad) {
            for (int k = 0; k < ORA_MAX_CONSTS; ++k) grad[p * ORA_MAX_CONSTS + k] = NAN;
            if (fit) fit[p] = NAN;
            if (bad == 2) rc = -2;
            continue;
        }
        double f = se / sw, scale = 1.0 / sw;
        if (metric == ORA_RMSE) {
            f = sqrt(f);
            scale = (f > 0.0) ? scale / (2.0 * f) : 0.0;
        }
        for (int k = 0; k < ORA_MAX_CONSTS; ++k)
            grad[p * ORA_MAX_CONSTS + k] = (k < nc) ? g[k] * scale : 0.0;
        if (fit) fit[p] = f;
    }
    return rc;
}

/* ---- Adam (Kingma & Ba 2015, Algorithm 1), one step on n parameters --- */
void ora_adam(double *theta, const double *g, double *m, double *v, int64_t n,
              int step, double lr, double beta1, double beta2, double eps) {
    double b1t = 1.0 - pow(beta1, (double)step);
    double b2t = 1.0 - pow(beta2, (double)step);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
        double mh = m[i] / b1t, vh = v[i] / b2t;
        theta[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* ---- mutation (Sec. II-A mutation kinds, Sec. III-C2 hoisted crossover) -- *
 * One offspring per index t.  Its random words come from one Philox4x32-10
 * stream: word k = Philox(counter = (k/4, t, offset lo32, offset hi32),
 * key = (seed lo32, seed hi32))[k%4], taken in order.  A word u picks an
 * index in [0, n) as (u * n) >> 32 and a kind by comparing u with the
 * cumulative thresholds floor(p * 2^32).
 *   kind      : crossover, subtree, hoist, point, else reproduction
 *   crossover : node i of the parent, node j of the donor (uniform); the
 *               child is the parent with subtree i replaced by donor
 *               subtree j; while the child holds more than 255 nodes or
 *               needs more than 20 stack slots, j moves to a node drawn
 *               uniformly among its proper descendants (the hoisted
 *               crossover of Sec. III-C2)
 *   subtree   : a random "grow" tree of the given depth is the donor
 *               (drawn first), then as crossover with j = its root
 *   hoist     : node i of the parent, then k among the proper descendants
 *               of i (k = i for a terminal); subtree i is replaced by
 *               subtree k
 *   point     : each node in prefix order is replaced with probability
 *               p_replace: a function by one of the allowed functions of
 *               the same arity, a terminal by a new terminal
 *   terminal  : one word picks f in [0, n_feat]; f < n_feat gives variable
 *               f, else a constant c = (w >> 8) * 2^-23 - 1 from the next
 *               word w (exact in float, uniform on [-1, 1))
 *   grow tree : a node at depth < limit is a terminal when a word picks
 *               one of the 2 terminal kinds among 2 + (allowed functions),
 *               else one of the allowed functions (uniform); nodes at the
 *               limit are terminals
 * A parent that is not a valid program is copied unchanged (kind
 * reproduction) when it has 1 to 255 nodes and replaced by the one-node
 * program 0 otherwise; an invalid donor turns a crossover into a
 * reproduction.  Returns 0, or -1 for bad arguments (a parent index out of
 * range among them). */
enum { ORA_MUT_REPRO = 0, ORA_MUT_CROSS = 1, ORA_MUT_SUBTREE = 2, ORA_MUT_HOIST = 3,
       ORA_MUT_POINT = 4 };

typedef struct {
    uint64_t seed, offset;
    int64_t t;
    uint32_t k;
} ora_stream;

static uint32_t stream_next(ora_stream *s) {
    uint32_t ctr[4] = {s->k >> 2, (uint32_t)s->t, (uint32_t)s->offset,
                       (uint32_t)(s->offset >> 32)};
    uint32_t key[2] = {(uint32_t)s->seed, (uint32_t)(s->seed >> 32)};
    uint32_t o[4];
    ora_philox4x32_10(ctr, key, o);
    uint32_t w = o[s->k & 3];
    s->k += 1;
    return w;
}

static int pick(ora_stream *s, int n) {
    return (int)(((uint64_t)stream_next(s) * (uint64_t)n) >> 32);
}

/* number of nodes of the subtree rooted at node i of a prefix list */
static int subtree_size(const ora_node *p, int len, int i) {
    int need = 1;
    for (int m = i; m < len; ++m) {
        need += ora_op_arity(p[m].op) - 1;
        if (need == 0) return m - i + 1;
    }
    return -1;
}

static ora_node new_terminal(ora_stream *s, int n_feat) {
    ora_node nd = {ORA_CONST, 0, 0.0f};
    int f = pick(s, n_feat + 1);
    if (f < n_feat) {
        nd.op = ORA_VAR;
        nd.feat = (int16_t)f;
    } else {
        uint32_t w = stream_next(s);
        nd.c = (float)(w >> 8) * 0x1p-23f - 1.0f;
    }
    return nd;
}

/* a grow tree of depth <= limit, in prefix order; returns its length */
static int grow_tree(ora_stream *s, int limit, const int *funcs, int nf, int n_feat,
                     ora_node *out) {
    int depth_of_slot[2 * ORA_MAX_LEN];
    int top = 0, n = 0;
    depth_of_slot[top++] = 0;
    while (top > 0) {
        int d = depth_of_slot[--top];
        int terminal = d >= limit || pick(s, nf + 2) < 2;
        if (terminal) {
            out[n++] = new_terminal(s, n_feat);
        } else {
            ora_node nd = {(int16_t)funcs[pick(s, nf)], 0, 0.0f};
            out[n++] = nd;
            for (int a = 0; a < ora_op_arity(nd.op); ++a) depth_of_slot[top++] = d + 1;
        }
    }
    return n;
}

/* parent with subtree [i, i+si) replaced by donor subtree [j, j+sj); the
 * child's length, or 0 when it exceeds 255 nodes or 20 stack slots */
static int splice(const ora_node *par, int lp, int i, int si, const ora_node *don, int j, int sj,
                  ora_node *out) {
    int len = i + sj + (lp - i - si);
    if (len > ORA_MAX_LEN) return 0;
    memcpy(out, par, (size_t)i * sizeof(ora_node));
    memcpy(out + i, don + j, (size_t)sj * sizeof(ora_node));
    memcpy(out + i + sj, par + i + si, (size_t)(lp - i - si) * sizeof(ora_node));
    int hw = 0;
    ora_validate(out, len, 1 << 15, &hw);
    return hw <= ORA_MAX_STACK ? len : 0;
}

/* hoisted crossover of donor subtree j into parent node i */
static int hoisted_splice(ora_stream *s, const ora_node *par, int lp, int i, const ora_node *don,
                          int ld, int j, ora_node *out) {
    int si = subtree_size(par, lp, i);
    int sj = subtree_size(don, ld, j);
    for (;;) {
        int len = splice(par, lp, i, si, don, j, sj, out);
        if (len > 0) return len;
        if (sj == 1) return 0; /* a terminal always fits a valid parent */
        j = j + 1 + pick(s, sj - 1);
        sj = subtree_size(don, ld, j);
    }
}

int ora_mutate(const ora_node *progs, const int32_t *offsets, int n_progs, int n_feat,
               const int32_t *parents, int n_out, const double probs[5], int subtree_depth,
               uint32_t funcs_mask, uint64_t seed, uint64_t offset, ora_node *out_nodes,
               int32_t *out_offsets, int32_t *out_kind) {
    int funcs[ORA_NOPS], nf = 0, f1[ORA_NOPS], n1 = 0, f2[ORA_NOPS], n2 = 0;
    for (int op = ORA_ADD; op < ORA_NOPS; ++op) {
        if (!(funcs_mask >> op & 1u)) continue;
        funcs[nf++] = op;
        if (ora_op_arity(op) == 1) f1[n1++] = op;
        else f2[n2++] = op;
    }
    if (nf == 0 || n_feat < 1 || subtree_depth < 0 || subtree_depth > 6) return -1;
    double cum = 0.0;
    uint64_t thr[4];
    for (int q = 0; q < 4; ++q) {
        if (!(probs[q] >= 0.0 && probs[q] <= 1.0)) return -1;
        cum += probs[q];
        double v = floor(cum * 4294967296.0);
        thr[q] = v >= 4294967296.0 ? 4294967296ull : (uint64_t)v;
    }
    if (cum > 1.0 + 1e-6 || !(probs[4] >= 0.0 && probs[4] <= 1.0)) return -1;
    double vr = floor(probs[4] * 4294967296.0);
    uint64_t thr_replace = vr >= 4294967296.0 ? 4294967296ull : (uint64_t)vr;
    for (int t = 0; t < 2 * n_out; ++t)
        if (parents[t] < 0 || parents[t] >= n_progs) return -1;

    ora_node child[ORA_MAX_LEN], tree[ORA_MAX_LEN];
    int32_t pos = 0;
    out_offsets[0] = 0;
    for (int t = 0; t < n_out; ++t) {
        ora_stream s = {seed, offset, t, 0};
        uint32_t u = stream_next(&s);
        int kind = ORA_MUT_REPRO;
        for (int q = 0; q < 4; ++q)
            if ((uint64_t)u < thr[q]) { kind = q + 1; break; }
        const ora_node *par = progs + offsets[parents[2 * t]];
        int lp = offsets[parents[2 * t] + 1] - offsets[parents[2 * t]];
        const ora_node *don = progs + offsets[parents[2 * t + 1]];
        int ld = offsets[parents[2 * t + 1] + 1] - offsets[parents[2 * t + 1]];
        if (ora_validate(par, lp, n_feat, NULL) != ORA_OK) {
            kind = ORA_MUT_REPRO;
            if (lp < 1 || lp > ORA_MAX_LEN) {
                static const ora_node zero = {ORA_CONST, 0, 0.0f};
                par = &zero;
                lp = 1;
            }
        }
        if (kind == ORA_MUT_CROSS && ora_validate(don, ld, n_feat, NULL) != ORA_OK)
            kind = ORA_MUT_REPRO;
        int len = 0;
        if (kind == ORA_MUT_CROSS) {
            int i = pick(&s, lp);
            int j = pick(&s, ld);
            len = hoisted_splice(&s, par, lp, i, don, ld, j, child);
        } else if (kind == ORA_MUT_SUBTREE) {
            int lt = grow_tree(&s, subtree_depth, funcs, nf, n_feat, tree);
            int i = pick(&s, lp);
            len = hoisted_splice(&s, par, lp, i, tree, lt, 0, child);
        } else if (kind == ORA_MUT_HOIST) {
            int i = pick(&s, lp);
            int si = subtree_size(par, lp, i);
            int k = si > 1 ? i + 1 + pick(&s, si - 1) : i;
            len = splice(par, lp, i, si, par, k, subtree_size(par, lp, k), child);
        } else if (kind == ORA_MUT_POINT) {
            memcpy(child, par, (size_t)lp * sizeof(ora_node));
            len = lp;
            for (int i = 0; i < lp; ++i) {
                if ((uint64_t)stream_next(&s) >= thr_replace) continue;
                int a = ora_op_arity(par[i].op);
                if (a == 0) {
                    child[i] = new_terminal(&s, n_feat);
                } else {
                    const int *same = a == 1 ? f1 : f2;
                    int ns = a == 1 ? n1 : n2;
                    if (ns > 0) {
                        ora_node nd = {(int16_t)same[pick(&s, ns)], 0, 0.0f};
                        child[i] = nd;
                    }
                }
            }
        }
        if (len == 0) { /* reproduction, or a splice that could not fit */
            memcpy(child, par, (size_t)lp * sizeof(ora_node));
            len = lp;
            kind = ORA_MUT_REPRO;
        }
        memcpy(out_nodes + pos, child, (size_t)len * sizeof(ora_node));
        pos += len;
        out_offsets[t + 1] = pos;
        if (out_kind) out_kind[t] = kind;
    }
    return 0;
}

int ora_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
