"""Pins of the CPU oracle against things other than itself (CPU only).

Each test ties an oracle function to a fact fixed by the paper or by
mathematics: hand-evaluated tiny programs, protected-operator point values,
closed forms, invariants between independent evaluation orders, library
routines (cuRAND's host Philox, scikit-learn metrics) and finite
differences.  A plausible mistake anywhere in the oracle (a swapped operand,
a dropped weight, a wrong sign in a derivative, a missing Philox round)
fails at least one of them.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np
import pytest

import oracle
from paper_2110_11226_gb300 import synth
from helpers import pack, parse_prefix, read_table

POINTS = [(1.5, -2.25), (0.75, 3.0), (-4.0, 0.5), (2.5, 1.25), (-0.375, -1.75)]


def _X(points):
    return np.array(points, np.float32).T.copy()  # [2][n]


# --------------------------------------------------------------------------
# evaluation order and operand order (Sec. III-A)
# --------------------------------------------------------------------------
def test_tiny_programs_brute_force():
    rows = read_table("tiny_programs.txt")
    assert len(rows) >= 50
    progs = [parse_prefix(r[0]) for r in rows]
    nodes, off = pack(progs)
    X = _X(POINTS)
    pred, st = oracle.predict64(nodes, off, X)
    assert (st == 0).all()
    p32 = oracle.predict32(nodes, off, X)
    for i, r in enumerate(rows):
        for j, (a, b) in enumerate(POINTS):
            x0, x1 = float(np.float32(a)), float(np.float32(b))
            want = eval(r[1], {"math": math, "abs": abs, "max": max, "min": min}, {"x0": x0, "x1": x1})
            assert pred[i, j] == want, (r[0], a, b, pred[i, j], want)
            # FP32 mode rounds each step: stays within float accuracy of it
            assert abs(float(p32[i, j]) - want) <= 1e-5 * max(1.0, abs(want)), r[0]


def _f32(x):
    return float(np.float32(x))


def test_protected_points():
    t = _f32(0.001)
    env = {"math": math, "t": t, "f32": _f32, "inf": math.inf}
    for op, a, b, want, _cite in read_table("protected_points.txt"):
        av = _f32(eval(a, env))
        prog = [(synth.OP[op], 0, 0.0), (synth.OP["var"], 0, 0.0)]
        cols = [av]
        if b != "-":
            prog.append((synth.OP["var"], 1, 0.0))
            cols.append(_f32(eval(b, env)))
        X = np.array(cols, np.float32).reshape(len(cols), 1)
        nodes, off = pack([prog])
        got = oracle.predict64(nodes, off, X)[0][0, 0]
        exp_v = float(eval(want, env))
        assert got == exp_v and math.copysign(1, got) == math.copysign(1, exp_v), (op, a, b, got, exp_v)
        g32 = float(oracle.predict32(nodes, off, X)[0, 0])
        if math.isinf(exp_v) or exp_v in (0.0, 1.0, 2.0):
            assert g32 == _f32(exp_v), (op, a, b, g32)
        else:
            assert abs(g32 - exp_v) <= 2 * abs(float(np.spacing(np.float32(exp_v)))), (op, a, b, g32)


# independent evaluators used only for the order invariants below
def _fn(name, a, b=None):
    thr = _f32(0.001)
    if name == "add": return a + b
    if name == "sub": return a - b
    if name == "mul": return a * b
    if name == "div": return 1.0 if abs(b) < thr else a / b
    if name == "sqrt": return math.sqrt(abs(a))
    if name == "log": return 0.0 if abs(a) < thr else math.log(abs(a))
    if name == "exp":
        try:
            return math.exp(a)
        except OverflowError:
            return math.inf
    if name == "sin": return math.sin(a) if math.isfinite(a) else math.nan
    if name == "cos": return math.cos(a) if math.isfinite(a) else math.nan
    if name == "tan": return math.tan(a) if math.isfinite(a) else math.nan
    if name == "abs": return abs(a)
    if name == "neg": return -a
    if name == "inv": return 0.0 if abs(a) < thr else 1.0 / a
    if name == "sq": return a * a
    if name == "cube": return (a * a) * a
    if name == "cbrt": return math.cbrt(a)
    if name == "tanh": return math.tanh(a)
    if name == "atan": return math.atan(a)
    if name in ("sinh", "cosh"):
        try:
            return math.sinh(a) if name == "sinh" else math.cosh(a)
        except OverflowError:
            return math.copysign(math.inf, a) if name == "sinh" else math.inf
    if name in ("max", "min"):
        if math.isnan(a) or math.isnan(b): return math.nan
        return (a if a > b else b) if name == "max" else (a if a < b else b)
    raise KeyError(name)


def _recursive(prog, x):
    pos = 0

    def rec():
        nonlocal pos
        op, feat, c = prog[pos]
        pos += 1
        name = synth.OP_NAME[op]
        if name == "const": return float(np.float32(c))
        if name == "var": return float(x[feat])
        if synth.ARITY[op] == 1: return _fn(name, rec())
        left = rec()
        right = rec()
        return _fn(name, left, right)

    return rec()


def _to_postfix(prog):
    """Children first (left, then right), then the parent."""
    pos = 0

    def rec():
        nonlocal pos
        node = prog[pos]
        pos += 1
        kids = [rec() for _ in range(synth.ARITY[node[0]])]
        return [n for k in kids for n in k] + [node]

    return rec()


def _postfix_eval(post, x):
    st = []
    for op, feat, c in post:
        name = synth.OP_NAME[op]
        if name == "const": st.append(float(np.float32(c)))
        elif name == "var": st.append(float(x[feat]))
        elif synth.ARITY[op] == 1: st.append(_fn(name, st.pop()))
        else:
            right = st.pop()
            left = st.pop()
            st.append(_fn(name, left, right))
    assert len(st) == 1
    return st[0]


def test_reverse_scan_matches_recursive_and_postfix():
    funcs = synth.EXTENDED_SET
    nodes, off = synth.random_programs(300, 7, funcs, 3, seed=7)
    rng = np.random.default_rng(3)
    X = rng.uniform(-3, 3, size=(3, 12)).astype(np.float32)
    pred, st = oracle.predict64(nodes, off, X)
    assert (st == 0).all()
    progs = synth.unpack(nodes, off)
    for i, prog in enumerate(progs):
        post = _to_postfix(prog)
        for r in range(X.shape[1]):
            x = X[:, r].astype(np.float64)
            a = _recursive(prog, x)
            b = _postfix_eval(post, x)
            c = pred[i, r]
            same = lambda u, v: (u == v) or (math.isnan(u) and math.isnan(v))
            assert same(a, c) and same(b, c), (i, r, a, b, c)


# --------------------------------------------------------------------------
# stack bound (Sec. III-C2: a stack of size m evaluates depth m-1)
# --------------------------------------------------------------------------
def _full_binary(depth):
    if depth == 0:
        return [(synth.OP["var"], 0, 0.0)]
    return [(synth.OP["add"], 0, 0.0)] + _full_binary(depth - 1) + _full_binary(depth - 1)


def _left_spine(depth):
    prog = []
    for _ in range(depth):
        prog.append((synth.OP["sub"], 0, 0.0))
    prog.append((synth.OP["var"], 0, 0.0))
    prog += [(synth.OP["const"], 0, 1.0)] * depth
    return prog


def test_high_water_of_full_tree_is_depth_plus_one():
    for d in range(0, 8):
        st, hw = oracle.validate(_full_binary(d), 1)
        assert st == oracle.OK and hw == d + 1
    # a left spine of depth d holds d+1 values at once (all right operands
    # wait while the left subtree is evaluated last)
    for d in range(1, 25):
        st, hw = oracle.validate(_left_spine(d), 1)
        assert hw == d + 1
        assert st == (oracle.OK if d + 1 <= 20 else oracle.TOO_DEEP)


def test_validate_errors():
    V, C_, A = synth.OP["var"], synth.OP["const"], synth.OP["add"]
    assert oracle.validate([(A, 0, 0), (V, 0, 0)], 1)[0] == oracle.UNDERFLOW
    assert oracle.validate([(V, 0, 0), (V, 0, 0)], 1)[0] == oracle.LEFTOVER
    assert oracle.validate([(99, 0, 0)], 1)[0] == oracle.BAD_OP
    assert oracle.validate([(V, 3, 0)], 3)[0] == oracle.BAD_FEATURE
    assert oracle.validate([(V, -1, 0)], 3)[0] == oracle.BAD_FEATURE
    assert oracle.validate(np.zeros(0, oracle.NODE_DTYPE), 1)[0] == oracle.BAD_LENGTH
    long = [(A, 0, 0), (C_, 0, 1.0)] * 127 + [(C_, 0, 1.0)]  # 255 nodes, right spine
    assert oracle.validate(long, 1)[0] == oracle.OK
    assert oracle.validate(long + [(C_, 0, 1.0)], 1)[0] == oracle.BAD_LENGTH


# --------------------------------------------------------------------------
# fitness: closed forms, invariants, library metrics (Sec. III-C3)
# --------------------------------------------------------------------------
def _rand_data(n, seed, binary=False):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-5, 5, size=(2, n)).astype(np.float32)
    if binary:
        y = (rng.random(n) < 0.4).astype(np.float32)
    else:
        y = rng.normal(1.0, 2.0, n).astype(np.float32)
    w = rng.uniform(0.5, 3.0, n).astype(np.float32)
    return X, y, w


def test_constant_program_closed_forms():
    X, y, w = _rand_data(501, 1)
    c = np.float32(0.625)
    nodes, off = pack([[(synth.OP["const"], 0, float(c))]])
    yd, wd = y.astype(np.float64), w.astype(np.float64)
    ybar = np.sum(wd * yd) / np.sum(wd)
    var_w = np.sum(wd * (yd - ybar) ** 2) / np.sum(wd)
    mse = oracle.fitness(nodes, off, X, y, w, "mse")[0][0]
    assert mse == pytest.approx(var_w + (ybar - float(c)) ** 2, rel=1e-12)
    rmse = oracle.fitness(nodes, off, X, y, w, "rmse")[0][0]
    assert rmse == pytest.approx(math.sqrt(var_w + (ybar - float(c)) ** 2), rel=1e-12)
    zero, zoff = pack([[(synth.OP["const"], 0, 0.0)]])
    mae0 = oracle.fitness(zero, zoff, X, y, w, "mae")[0][0]
    assert mae0 == pytest.approx(np.sum(wd * np.abs(yd)) / np.sum(wd), rel=1e-12)
    rmse0 = oracle.fitness(zero, zoff, X, y, None, "rmse")[0][0]
    assert rmse0 == pytest.approx(math.sqrt(np.mean(yd ** 2)), rel=1e-12)
    Xb, yb, wb = _rand_data(333, 2, binary=True)
    ll0 = oracle.fitness(zero, zoff, Xb, yb, wb, "logloss")[0][0]
    assert ll0 == pytest.approx(math.log(2.0), rel=1e-15)


def _pagie_program(c1=1.0):
    def term(f):
        sq = [(synth.OP["mul"], 0, 0.0), (synth.OP["var"], f, 0.0), (synth.OP["var"], f, 0.0)]
        x4 = [(synth.OP["mul"], 0, 0.0)] + sq + sq
        return [(synth.OP["div"], 0, 0.0)] + x4 + [(synth.OP["add"], 0, 0.0),
                                                   (synth.OP["const"], 0, c1)] + x4
    return [(synth.OP["add"], 0, 0.0)] + term(0) + term(1)


def test_exact_pagie_program():
    d = synth.pagie_data(4096, 5)
    nodes, off = pack([_pagie_program()])
    pred = oracle.predict64(nodes, off, d.X)[0][0]
    x = d.X.astype(np.float64)
    closed = 1.0 / (1.0 + x[0] ** -4.0) + 1.0 / (1.0 + x[1] ** -4.0)  # Eq. pagie
    ok = (x[0] != 0) & (x[1] != 0)
    np.testing.assert_allclose(pred[ok], closed[ok], rtol=4e-15)
    mse = oracle.fitness(nodes, off, d.X, d.y, None, "mse")[0][0]
    # y is stored in float32: only its rounding (<= 2^-24 |y|, |y| < 2) remains
    assert mse <= (2.0 * 2.0 ** -24) ** 2
    assert mse > 0.0


def test_metric_invariants():
    X, y, w = _rand_data(257, 3)
    nodes, off = synth.ramped_half_and_half(40, 2, 5, synth.FULL_SET, 2, seed=11)
    for m in ("mae", "mse", "rmse"):
        f1 = oracle.fitness(nodes, off, X, y, w, m)[0]
        f2 = oracle.fitness(nodes, off, X, y, w * np.float32(4.0), m)[0]
        np.testing.assert_allclose(f1, f2, rtol=1e-13)
        # duplicating row 0 equals doubling its weight
        X2 = np.concatenate([X, X[:, :1]], axis=1)
        y2 = np.concatenate([y, y[:1]])
        w2 = np.concatenate([w, w[:1]])
        wd = w.copy()
        wd[0] *= 2
        f3 = oracle.fitness(nodes, off, X2, y2, w2, m)[0]
        f4 = oracle.fitness(nodes, off, X, y, wd, m)[0]
        np.testing.assert_allclose(f3, f4, rtol=1e-12)
    mse = oracle.fitness(nodes, off, X, y, w, "mse")[0]
    rmse = oracle.fitness(nodes, off, X, y, w, "rmse")[0]
    fin = np.isfinite(mse)
    np.testing.assert_allclose(rmse[fin] ** 2, mse[fin], rtol=1e-13)
    # unit weights == unweighted numpy mean of the oracle's own residuals
    pred = oracle.predict64(nodes, off, X)[0]
    un = oracle.fitness(nodes, off, X, y, None, "mae")[0]
    np.testing.assert_allclose(un, np.mean(np.abs(pred - y.astype(np.float64)), axis=1), rtol=1e-12)


def test_metrics_match_scikit_learn():
    sk = pytest.importorskip("sklearn.metrics")
    X, y, w = _rand_data(300, 4)
    nodes, off = synth.ramped_half_and_half(20, 2, 4, synth.BASIC_SET, 2, seed=12)
    pred = oracle.predict64(nodes, off, X)[0]
    mse = oracle.fitness(nodes, off, X, y, w, "mse")[0]
    mae = oracle.fitness(nodes, off, X, y, w, "mae")[0]
    for i in range(len(mse)):
        if not np.all(np.isfinite(pred[i])) or np.max(np.abs(pred[i])) > 1e100:
            continue
        assert mse[i] == pytest.approx(sk.mean_squared_error(y, pred[i], sample_weight=w), rel=1e-9)
        assert mae[i] == pytest.approx(sk.mean_absolute_error(y, pred[i], sample_weight=w), rel=1e-9)
    Xb, yb, wb = _rand_data(300, 5, binary=True)
    bn, boff = synth.ramped_half_and_half(20, 2, 4, ("add", "sub", "mul", "sin"), 2, seed=13)
    pb = oracle.predict64(bn, boff, Xb)[0]
    ll = oracle.fitness(bn, boff, Xb, yb, wb, "logloss")[0]
    for i in range(len(ll)):
        if np.max(np.abs(pb[i])) > 8:  # log(1 - sigmoid) loses digits in sklearn beyond this
            continue
        prob = 1.0 / (1.0 + np.exp(-pb[i]))
        ref = sk.log_loss(yb, prob, sample_weight=wb, labels=[0.0, 1.0])
        assert ll[i] == pytest.approx(ref, rel=1e-9)


def test_pearson_closed_forms_and_numpy():
    """Weighted Pearson fitness |r|: an affine image of y scores exactly 1
    whatever its sign, a constant scores 0, unit weights give numpy's
    corrcoef, integer weights equal duplicated rows, and rescaling the
    weights or the prediction changes nothing."""
    rng = np.random.default_rng(21)
    n = 777
    X = rng.uniform(-3, 3, size=(2, n)).astype(np.float32)
    y = X[0].copy()  # y = x0 exactly
    w = rng.uniform(0.5, 2.0, n).astype(np.float32)
    progs = [
        [(synth.OP["add"], 0, 0.0), (synth.OP["mul"], 0, 0.0), (synth.OP["const"], 0, 2.5),
         (synth.OP["var"], 0, 0.0), (synth.OP["const"], 0, 1.0)],       # 2.5 x0 + 1
        [(synth.OP["neg"], 0, 0.0), (synth.OP["var"], 0, 0.0)],          # -x0
        [(synth.OP["const"], 0, 0.375)],                                 # constant
        [(synth.OP["sin"], 0, 0.0), (synth.OP["var"], 1, 0.0)],          # unrelated
    ]
    nodes, off = pack(progs)
    f = oracle.fitness(nodes, off, X, y, w, "pearson")[0]
    assert f[0] == pytest.approx(1.0, abs=1e-14) and f[1] == pytest.approx(1.0, abs=1e-14)
    assert f[2] == 0.0
    assert f[3] < 0.2
    # unit weights: numpy's (unweighted) correlation of the oracle's predictions
    Xr, yr, wr = _rand_data(401, 6)
    rn, roff = synth.ramped_half_and_half(30, 2, 5, synth.FULL_SET, 2, seed=14)
    pred = oracle.predict64(rn, roff, Xr)[0]
    un = oracle.fitness(rn, roff, Xr, yr, None, "pearson")[0]
    for i in range(len(un)):
        if not np.all(np.isfinite(pred[i])) or np.ptp(pred[i]) == 0:
            continue
        assert un[i] == pytest.approx(abs(np.corrcoef(pred[i], yr.astype(np.float64))[0, 1]),
                                      rel=1e-10, abs=1e-13)
    # integer weights == duplicated rows; scaled weights change nothing
    wi = rng.integers(1, 4, size=len(yr)).astype(np.float32)
    rep = np.repeat(np.arange(len(yr)), wi.astype(int))
    fw = oracle.fitness(rn, roff, Xr, yr, wi, "pearson")[0]
    fd = oracle.fitness(rn, roff, Xr[:, rep], yr[rep], None, "pearson")[0]
    fs = oracle.fitness(rn, roff, Xr, yr, wi * np.float32(8.0), "pearson")[0]
    fin = np.isfinite(fw)
    np.testing.assert_allclose(fw[fin], fd[fin], rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(fw[fin], fs[fin], rtol=1e-12, atol=1e-14)
    # prediction scaled by -3 (a wrapped program): same |r|
    scaled = []
    for prog in synth.unpack(rn, roff):
        scaled.append([(synth.OP["mul"], 0, 0.0), (synth.OP["const"], 0, -3.0)] + list(prog))
    sn, soff = pack(scaled)
    f3 = oracle.fitness(sn, soff, Xr, yr, wr, "pearson")[0]
    f1 = oracle.fitness(rn, roff, Xr, yr, wr, "pearson")[0]
    ok = np.isfinite(f1) & np.isfinite(f3) & (f1 > 1e-6)
    np.testing.assert_allclose(f3[ok], f1[ok], rtol=1e-9)


def test_spearman_matches_scipy_and_closed_forms():
    """Spearman fitness |r_s| = |Pearson of the average ranks|: scipy's
    rankdata and spearmanr (library routines) on the oracle's predictions,
    with ties; 1 for any strictly monotone image of y, 0 for a constant;
    weights scaled by a constant change nothing."""
    st = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(31)
    v = np.round(rng.normal(size=500), 1)  # many ties
    np.testing.assert_array_equal(oracle.average_ranks(v), st.rankdata(v))
    n = 600
    X = rng.uniform(-2, 2, size=(2, n)).astype(np.float32)
    X[1, :150] = np.round(X[1, :150])  # ties in a feature
    y = X[0].copy()
    progs = [
        [(synth.OP["exp"], 0, 0.0), (synth.OP["var"], 0, 0.0)],            # monotone up
        [(synth.OP["neg"], 0, 0.0), (synth.OP["var"], 0, 0.0)],            # monotone down
        [(synth.OP["const"], 0, 0.5)],                                     # constant
    ]
    nodes, off = pack(progs)
    f = oracle.fitness(nodes, off, X, y, None, "spearman")[0]
    assert f[0] == pytest.approx(1.0, abs=1e-14) and f[1] == pytest.approx(1.0, abs=1e-14)
    assert f[2] == 0.0
    Xr, yr, wr = _rand_data(401, 6)
    yr[:60] = np.round(yr[:60])  # ties in y
    rn, roff = synth.ramped_half_and_half(30, 2, 5, synth.FULL_SET, 2, seed=15)
    pred = oracle.predict64(rn, roff, Xr)[0]
    un = oracle.fitness(rn, roff, Xr, yr, None, "spearman")[0]
    checked = 0
    for i in range(len(un)):
        if np.isnan(pred[i]).any() or np.ptp(pred[i]) == 0:
            continue
        want = abs(st.spearmanr(pred[i], yr.astype(np.float64)).statistic)
        assert un[i] == pytest.approx(want, rel=1e-10, abs=1e-13)
        checked += 1
    assert checked > 15
    f1 = oracle.fitness(rn, roff, Xr, yr, wr, "spearman")[0]
    f2 = oracle.fitness(rn, roff, Xr, yr, wr * np.float32(4.0), "spearman")[0]
    fin = np.isfinite(f1)
    np.testing.assert_allclose(f1[fin], f2[fin], rtol=1e-12, atol=1e-14)


def test_logloss_limits():
    # the c*|p| term vanishes for the matching label, so saturated correct
    # predictions cost 0 and saturated wrong ones cost |p|
    assert oracle.loss("logloss", math.inf, 1.0) == 0.0
    assert oracle.loss("logloss", -math.inf, 0.0) == 0.0
    assert oracle.loss("logloss", math.inf, 0.0) == math.inf
    assert oracle.loss("logloss", 50.0, 0.0) == pytest.approx(50.0, rel=1e-15)
    assert math.isnan(oracle.loss("logloss", math.nan, 1.0))
    for p in (-3.0, -0.5, 0.0, 0.7, 4.0):
        for yy in (0.0, 1.0):
            s = 1.0 / (1.0 + math.exp(-p))
            ref = -(yy * math.log(s) + (1 - yy) * math.log(1 - s))
            assert oracle.loss("logloss", p, yy) == pytest.approx(ref, rel=1e-13)


def test_fp32_mode_matches_numpy_float32():
    # add/sub/mul/div/sqrt/abs/neg are correctly rounded in IEEE single:
    # numpy float32 arithmetic in the same order gives the same bits
    rng = np.random.default_rng(9)
    X = rng.uniform(-4, 4, size=(2, 1000)).astype(np.float32)
    progs = ["sub div x0 x1 mul x1 x0", "add sqrt sub x0 x1 neg abs x0",
             "div div x0 x1 add x1 0.75", "mul sub x0 0.3 sub x1 0.3"]
    nodes, off = pack([parse_prefix(p) for p in progs])
    got = oracle.predict32(nodes, off, X)
    x0, x1 = X[0], X[1]
    thr = np.float32(0.001)
    pdiv = lambda a, b: np.where(np.abs(b) < thr, np.float32(1), a / np.where(np.abs(b) < thr, np.float32(1), b)).astype(np.float32)
    with np.errstate(all="ignore"):
        want = [pdiv(x0, x1) - x1 * x0,
                np.sqrt(np.abs(x0 - x1)) + (-np.abs(x0)),
                pdiv(pdiv(x0, x1), x1 + np.float32(0.75)),
                (x0 - np.float32(0.3)) * (x1 - np.float32(0.3))]
    for i in range(len(progs)):
        np.testing.assert_array_equal(got[i], np.asarray(want[i], np.float32))


@pytest.mark.parametrize("funcs", [synth.FULL_SET + ("tan",), synth.EXTENDED_SET])
def test_error_bound_covers_fp32_evaluation(funcs):
    nodes, off = synth.ramped_half_and_half(400, 2, 7, funcs, 2, seed=21)
    X = synth.pagie_data(2000, 22).X
    v, e, fl = oracle.predict_bound(nodes, off, X, ulps_fn=4.0)
    p32 = oracle.predict32(nodes, off, X).astype(np.float64)
    ok = (fl == 0) & np.isfinite(v) & np.isfinite(e)
    assert ok.mean() > 0.8
    with np.errstate(invalid="ignore"):  # inf - inf on rows outside `ok`
        err = np.abs(p32 - v)
    # first-order bound; 1.5 covers the neglected second-order terms
    bad = ok & (err > 1.5 * e + 1e-300)
    assert bad.sum() == 0, (np.argwhere(bad)[:5], err[bad][:5], e[bad][:5])
    # and it is not vacuous: most rows are certified to 1e-5 relative
    tight = ok & (e <= 2.5e-6 * np.abs(v))
    assert tight.sum() > 0.5 * ok.sum()


# --------------------------------------------------------------------------
# Philox4x32-10 and tournament selection (Sec. III-B, III-C1)
# --------------------------------------------------------------------------
def _curand():
    for path in ("/usr/local/cuda/lib64/libcurand.so",
                 "/usr/local/cuda/targets/sbsa-linux/lib/libcurand.so",
                 "libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(path)
        except OSError:
            continue
    return None


def test_philox_matches_curand_host_generator():
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not loadable")
    PHILOX = 161  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    for seed in (0, 42, 0x0123456789ABCDEF, 2 ** 64 - 1):
        gen = ctypes.c_void_p()
        assert lib.curandCreateGeneratorHost(ctypes.byref(gen), PHILOX) == 0
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_uint64(seed)) == 0
        n = 64
        out = np.zeros(n, np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
        lib.curandDestroyGenerator(gen)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        # cuRAND's host generator emits block b from counter (0, 0, b, 0)
        mine = np.concatenate([oracle.philox4x32_10([0, 0, b, 0], key) for b in range(n // 4)])
        np.testing.assert_array_equal(mine, out)


def test_tournament_draws_are_curand_philox_words():
    """Draw j of tournament 0 at offset b is word j % 4 of the Philox4x32-10
    block at counter (j / 4, 0, b, 0), mapped to [0, n) as (u * n) >> 32
    (Sec. III-B, III-C1).  cuRAND's host generator emits the block of counter
    (c0, 0, c2, 0) at position 65536 * c0 + c2 of its stream (asserted first),
    so the draws are pinned to the library's own words."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not loadable")
    PHILOX = 161  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    seed = 0x0123456789ABCDEF
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), PHILOX) == 0
    assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_uint64(seed)) == 0
    out = np.zeros(4 * (65536 + 64), np.uint32)
    assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(out.size)) == 0
    lib.curandDestroyGenerator(gen)
    blocks = out.reshape(-1, 4)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for c0 in (0, 1):
        for b in (0, 1, 63):
            np.testing.assert_array_equal(oracle.philox4x32_10([c0, 0, b, 0], key),
                                          blocks[65536 * c0 + b])
    for n in (7, 97, 1000, 2 ** 31 - 1):
        for b in range(64):
            for j in range(8):
                u = int(blocks[65536 * (j >> 2) + b][j & 3])
                assert oracle.tournament_draw(seed, b, 0, j, n) == (u * n) >> 32


def test_tournament_draws_uniform():
    n, T = 37, 20000
    draws = np.array([oracle.tournament_draw(42, 0, t, j, n) for t in range(T // 20) for j in range(20)])
    assert draws.min() >= 0 and draws.max() < n
    counts = np.bincount(draws, minlength=n)
    chi2 = np.sum((counts - T / n) ** 2 / (T / n))
    assert chi2 < 80.0  # chi^2 with 36 dof: p ~ 5e-5


def test_tournament_properties():
    n, T = 97, 300
    rng = np.random.default_rng(0)
    f = rng.normal(size=n).astype(np.float32)
    draws = lambda t, k: [oracle.tournament_draw(42, 0, t, j, n) for j in range(k)]
    w1 = oracle.tournament(f, T, 1, 42)
    assert all(w1[t] == draws(t, 1)[0] for t in range(T))
    const = np.full(n, 0.5, np.float32)
    wc = oracle.tournament(const, T, 20, 42)
    assert all(wc[t] == draws(t, 20)[0] for t in range(T))
    ident = np.arange(n, dtype=np.float32)
    wi = oracle.tournament(ident, T, 20, 42)
    assert all(wi[t] == min(draws(t, 20)) for t in range(T))
    wg = oracle.tournament(ident, T, 20, 42, greater_is_better=True)
    assert all(wg[t] == max(draws(t, 20)) for t in range(T))
    # parsimony (Eqs. parsimony, fitness): brute force over the draw list
    lens = rng.integers(3, 255, n).astype(np.int32)
    wp = oracle.tournament(f, T, 10, 7, lengths=lens, parsimony=0.01)
    for t in range(T):
        ds = [oracle.tournament_draw(7, 0, t, j, n) for j in range(10)]
        adj = [np.float64(f[i]) + 0.01 * np.float64(np.float32(0.01)) / 0.01 * lens[i] for i in ds]
        best = ds[int(np.argmin(adj))]
        assert wp[t] == best
    # NaN is the worst fitness
    fn = f.copy()
    fn[::2] = np.nan
    wn = oracle.tournament(fn, T, 20, 3)
    for t in range(T):
        ds = [oracle.tournament_draw(3, 0, t, j, n) for j in range(20)]
        finite = [i for i in ds if np.isfinite(fn[i])]
        if finite:
            assert np.isfinite(fn[wn[t]]) and fn[wn[t]] == min(fn[i] for i in finite)
    # the offset moves to a disjoint counter range
    assert not np.array_equal(oracle.tournament(f, T, 20, 42, offset=1), oracle.tournament(f, T, 20, 42))


# --------------------------------------------------------------------------
# constant gradients (reverse mode) and Adam
# --------------------------------------------------------------------------
def test_const_grad_closed_forms():
    X, y, w = _rand_data(400, 6)
    yd, wd = y.astype(np.float64), w.astype(np.float64)
    c = 0.8125
    nodes, off = pack([[(synth.OP["const"], 0, c)],
                       parse_prefix(f"mul {c} x0")])
    g, fit = oracle.const_grad(nodes, off, X, y, w, "mse")
    ybar = np.sum(wd * yd) / np.sum(wd)
    assert g[0, 0] == pytest.approx(2 * (c - ybar), rel=1e-12)
    x0 = X[0].astype(np.float64)
    assert g[1, 0] == pytest.approx(2 * np.sum(wd * (c * x0 - yd) * x0) / np.sum(wd), rel=1e-12)
    assert np.all(g[:, 1:] == 0)
    f_ref = oracle.fitness(nodes, off, X, y, w, "mse")[0]
    np.testing.assert_array_equal(fit, f_ref)
    # magnitude output: sum of |w 2 (c - y)| / sum w for the constant program
    _, _, ga = oracle.const_grad(nodes, off, X, y, w, "mse", with_abs=True)
    assert ga[0, 0] == pytest.approx(np.sum(wd * 2 * np.abs(c - yd)) / np.sum(wd), rel=1e-12)
    assert np.all(ga >= np.abs(g) * (1 - 1e-12))


@pytest.mark.parametrize("metric", ["mse", "rmse", "mae", "logloss"])
def test_const_grad_matches_central_differences(metric):
    binary = metric == "logloss"
    X, y, w = _rand_data(64, 8, binary=binary)
    funcs = synth.EXTENDED_SET
    nodes, off = synth.ramped_half_and_half(150, 2, 4, funcs, 2, seed=31, max_consts=16,
                                            const_range=(-2.0, 2.0))
    g, fit = oracle.const_grad(nodes, off, X, y, w, metric)
    checked = skipped = 0
    for p in range(len(off) - 1):
        seg = np.arange(off[p], off[p + 1])
        kidx = seg[nodes["op"][seg] == synth.OP["const"]]
        for k, node in enumerate(kidx):
            def f_at(h):
                nn = nodes.copy()
                nn["c"][node] = np.float32(nodes["c"][node] + h)
                return (oracle.fitness(nn, off, X, y, w, metric)[0][p],
                        float(nn["c"][node]))
            fp, cp = f_at(1e-3)
            fm, cm = f_at(-1e-3)
            fp2, cp2 = f_at(5e-4)
            fm2, cm2 = f_at(-5e-4)
            if not all(np.isfinite([fp, fm, fp2, fm2])):
                skipped += 1
                continue
            d1 = (fp - fm) / (cp - cm)
            d2 = (fp2 - fm2) / (cp2 - cm2)
            scale = max(abs(d2), abs(g[p, k]), 1e-6)
            if abs(d1 - d2) > 1e-4 * scale:  # not smooth over [c-h, c+h]
                skipped += 1
                continue
            # FD cannot resolve a slope below its own roundoff eps*|f|/h
            if 4 * np.finfo(float).eps * abs(fit[p]) / (cp2 - cm2) > 1e-6 * scale:
                skipped += 1
                continue
            assert abs(g[p, k] - d2) <= 1e-5 * scale + 2 * abs(d1 - d2), (p, k, g[p, k], d2, d1)
            checked += 1
    assert checked >= 80 and checked >= 3 * skipped, (checked, skipped)


def test_const_grad_rejects_more_than_16_constants():
    prog = parse_prefix(" ".join(["add"] * 16 + ["0.5"] * 17))
    nodes, off = pack([prog, parse_prefix("add x0 0.5")])
    X, y, w = _rand_data(10, 9)
    g, fit = oracle.const_grad(nodes, off, X, y, w, "mse")
    assert np.all(np.isnan(g[0])) and np.isfinite(g[1, 0])


def test_adam_constant_gradient_closed_form():
    # with a constant gradient g the bias-corrected moments are exactly g
    # and g^2, so every step moves by -lr * g / (|g| + eps) (Kingma & Ba)
    g = np.array([0.3, -2.0, 1e-3, 5.0])
    th = np.zeros(4)
    m = np.zeros(4)
    v = np.zeros(4)
    for t in range(1, 6):
        before = th.copy()
        oracle.adam(th, g, m, v, t, lr=1e-2)
        np.testing.assert_allclose(th - before, -1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-9)


# --------------------------------------------------------------------------
# the FP32 reverse mode (every per-row operation in float, sums in FP64):
# the yardstick the device adjoint is held to where FP32 rounding moves a
# gradient far from the FP64 one
# --------------------------------------------------------------------------
EPS32 = float(np.finfo(np.float32).eps)


def test_const_grad32_closed_forms():
    X, y, w = _rand_data(700, 12)
    yd, wd = y.astype(np.float64), w.astype(np.float64)
    sw = np.sum(wd)
    c = 0.8125  # exact in float
    nodes, off = pack([[(synth.OP["const"], 0, c)], parse_prefix(f"mul {c} x0")])
    x0 = X[0].astype(np.float64)
    # MSE: 2 (c - ybar_w) for the constant, 2 sum w (c x0 - y) x0 / sum w
    # for c x0; each row's term is a few float roundings off its exact value
    g, fit = oracle.const_grad32(nodes, off, X, y, w, "mse")
    rows = 2 * wd * (c - yd)
    assert abs(g[0, 0] - rows.sum() / sw) <= 4 * EPS32 * np.abs(rows).sum() / sw
    rows = 2 * wd * (c * x0 - yd) * x0
    assert abs(g[1, 0] - rows.sum() / sw) <= 6 * EPS32 * np.abs(rows).sum() / sw
    assert np.all(g[:, 1:] == 0)
    # RMSE: the MSE gradient over 2 RMSE
    g, fit = oracle.const_grad32(nodes[:1], off[:2], X, y, w, "rmse")
    rmse = math.sqrt(np.sum(wd * (yd - c) ** 2) / sw)
    assert fit[0] == pytest.approx(rmse, rel=1e-6)
    assert g[0, 0] == pytest.approx((c - np.sum(wd * yd) / sw) / rmse, rel=1e-5)
    # MAE: the weighted mean of sign(c - y)
    g, _ = oracle.const_grad32(nodes[:1], off[:2], X, y, w, "mae")
    assert g[0, 0] == pytest.approx(np.sum(wd * np.sign(c - yd)) / sw, rel=1e-12, abs=1e-12)
    # log-loss of sigmoid(c): sigma(c) - ybar_w
    Xb, yb, wb = _rand_data(500, 13, binary=True)
    g, fit = oracle.const_grad32(nodes[:1], off[:2], Xb, yb, wb, "logloss")
    ybw = np.sum(wb.astype(np.float64) * yb) / np.sum(wb.astype(np.float64))
    assert g[0, 0] == pytest.approx(1.0 / (1.0 + math.exp(-c)) - ybw, rel=1e-5)


def _fitness_of_fp32_predictions(nodes, off, X, y, w, metric):
    """Fitness of the oracle's FP32 predictions, the loss and sums in FP64."""
    p32 = oracle.predict32(nodes, off, X)
    p = p32.astype(np.float64)
    yd, wd = y.astype(np.float64), w.astype(np.float64)
    with np.errstate(all="ignore"):
        # a squared error beyond the float range makes the FP32 fitness
        # infinite: there is no slope to compare
        if metric in ("mse", "rmse") and not np.all(np.isfinite((p32 - y) * (p32 - y))):
            return np.full(p.shape[0], np.inf)
        if metric in ("mse", "rmse"):
            l = (p - yd) ** 2
        elif metric == "mae":
            l = np.abs(p - yd)
        else:
            l = np.logaddexp(0.0, p) - yd * p
        f = (l * wd).sum(axis=1) / wd.sum()
    return np.sqrt(f) if metric == "rmse" else f


@pytest.mark.parametrize("metric", ["mse", "rmse", "mae", "logloss"])
def test_const_grad32_matches_central_differences_of_fp32_fitness(metric):
    # the FP32 adjoint against difference quotients of a fitness built from
    # the FP32 forward evaluation (predict32), not from the adjoint's own
    # forward pass
    X, y, w = _rand_data(2000, 14, binary=metric == "logloss")
    nodes, off = synth.ramped_half_and_half(200, 2, 4, synth.FULL_SET + ("tan",), 2, seed=33,
                                            max_consts=16, const_range=(-2.0, 2.0))
    g, _ = oracle.const_grad32(nodes, off, X, y, w, metric)
    g64, _ = oracle.const_grad(nodes, off, X, y, w, metric)
    # MAE's slope jumps wherever a row's prediction crosses its target, so
    # its quotients take a narrower step
    h = 2e-4 if metric == "mae" else 2e-3
    checked = skipped = 0
    for p in range(len(off) - 1):
        seg = np.arange(off[p], off[p + 1])
        sub = nodes[seg].copy()
        soff = np.array([0, len(seg)], np.int32)
        kidx = np.flatnonzero(sub["op"] == synth.OP["const"])
        for k, node in enumerate(kidx):
            def f_at(h):
                nn = sub.copy()
                nn["c"][node] = np.float32(sub["c"][node] + h)
                return _fitness_of_fp32_predictions(nn, soff, X, y, w, metric)[0], float(nn["c"][node])
            fp, cp = f_at(2 * h)
            fm, cm = f_at(-2 * h)
            fp2, cp2 = f_at(h)
            fm2, cm2 = f_at(-h)
            if not all(np.isfinite([fp, fm, fp2, fm2])):
                skipped += 1
                continue
            d1 = (fp - fm) / (cp - cm)
            d2 = (fp2 - fm2) / (cp2 - cm2)
            scale = max(abs(d1), abs(d2), 1e-4)
            if abs(d1 - d2) > 1e-3 * scale:  # not smooth over [c-h, c+h]
                skipped += 1
                continue
            # the same quotient of the FP64 fitness: where the two disagree,
            # FP32 rounding (a constant absorbed by a much larger operand)
            # hides the slope from the FP32 quotient
            nn = sub.copy()
            nn["c"][node] = np.float32(cp2)
            q64p = oracle.fitness(nn, soff, X, y, w, metric)[0][0]
            nn["c"][node] = np.float32(cm2)
            q64m = oracle.fitness(nn, soff, X, y, w, metric)[0][0]
            d64 = (q64p - q64m) / (cp2 - cm2)
            if not np.isfinite(d64) or abs(d64 - d2) > 1e-3 * max(scale, abs(d64)):
                skipped += 1
                continue
            # and where even the FP64 quotient misses the FP64 reverse mode
            # (pinned above to FP64 differences and closed forms), a value
            # swamps the constant's effect at this step: no slope to see
            if abs(d64 - g64[p, k]) > 1e-3 * max(abs(d64), abs(g64[p, k]), 1e-4):
                skipped += 1
                continue
            assert abs(g[p, k] - d2) <= 2e-3 * scale + 4 * abs(d1 - d2), (p, k, g[p, k], d2, d1)
            checked += 1
    assert checked >= 80 and checked >= 2 * skipped, (checked, skipped)


@pytest.mark.parametrize("metric", ["mse", "rmse", "mae", "logloss"])
def test_const_grad32_agrees_with_fp64_reverse_mode_on_certified_programs(metric):
    # Where the FP32 error bound certifies every row of a program to 1e-5
    # (no protected-operator decision can flip), FP32 rounding moves each
    # per-row contribution by a few ulps; the sum then differs from the FP64
    # gradient by far less than 1e-5 of the sum of |contributions| (measured
    # about 7e-7 at most).  A wrong derivative rule moves it by a fraction of
    # that sum itself.
    rng = np.random.default_rng(15)
    n = 1500
    X = rng.uniform(-5, 5, size=(2, n)).astype(np.float32)
    if metric == "logloss":
        y = (rng.random(n) < 0.4).astype(np.float32)
    else:
        y = rng.normal(1.0, 2.0, n).astype(np.float32)
    w = rng.uniform(0.5, 3.0, n).astype(np.float32)
    nodes, off = synth.ramped_half_and_half(300, 2, 5, synth.FULL_SET, 2, seed=41, max_consts=16,
                                            const_range=(-2.0, 2.0))
    g64, _, gabs = oracle.const_grad(nodes, off, X, y, w, metric, with_abs=True)
    g32, f32 = oracle.const_grad32(nodes, off, X, y, w, metric)
    v, e, fl = oracle.predict_bound(nodes, off, X)
    with np.errstate(invalid="ignore"):
        cert = np.all((fl == 0) & np.isfinite(v) & (e <= 1e-5 * np.maximum(np.abs(v), 1e-30)),
                      axis=1)
    cert &= np.all(np.isfinite(g64), axis=1)
    assert cert.sum() >= 120
    # the certified programs cover every function of the set under a constant
    names = set()
    for p in np.flatnonzero(cert):
        seg = nodes["op"][off[p]:off[p + 1]]
        if (seg == synth.OP["const"]).any():
            names |= {synth.OP_NAME[int(o)] for o in seg}
    assert set(synth.FULL_SET) <= names, set(synth.FULL_SET) - names
    with np.errstate(invalid="ignore"):  # inf - inf outside the certified programs
        bad = cert[:, None] & (np.abs(g32 - g64) > 1e-5 * gabs + 1e-300)
    assert not bad.any(), (np.argwhere(bad)[:5], g32[bad][:5], g64[bad][:5])
    f64 = oracle.fitness(nodes, off, X, y, w, metric)[0]
    np.testing.assert_allclose(f32[cert], f64[cert], rtol=1e-5)
