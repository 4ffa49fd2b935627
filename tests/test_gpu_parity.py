"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Small cases run in full (several row tiles, a ragged tail, every metric);
the full-size workloads run in the launch configuration of bench.py and are
checked on sampled programs the oracle evaluates over every row.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_2110_11226_gb300 import gp, synth
from helpers import pack, parse_prefix, read_table
from parity import check_fitness, check_fitness_sampled, check_pearson, check_points

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def put(nodes, off, X, y=None, w=None):
    return (gp.nodes_to_device(nodes), dev(off.astype(np.int32)), dev(X),
            None if y is None else dev(y), None if w is None else dev(w))


def _weights(n, seed):
    return np.random.default_rng(seed).uniform(0.25, 4.0, n).astype(np.float32)


# --------------------------------------------------------------------------
# per-point values
# --------------------------------------------------------------------------
def test_predict_bit_exact_on_ieee_operators():
    """add/sub/mul/div/inv/sqrt/abs/neg/sq/cube/max/min are correctly rounded
    (or exact) on both sides and nothing is contracted into FMA: the GPU values equal the oracle's
    FP32 mode bit for bit (pagie_small programs and hand-written ones)."""
    wl = synth.workload("pagie_small")
    extra = synth.unpack(*synth.random_programs(300, 9, ("add", "sub", "mul", "div", "inv",
                                                         "sqrt", "abs", "neg", "sq", "cube",
                                                         "max", "min"), 2, seed=17))
    progs = synth.unpack(wl.nodes, wl.offsets) + extra
    nodes, off = pack(progs)
    for n in (4096, 4096 + 37, 5):
        X = synth.pagie_data(n, 3).X
        pn, po, dX, _, _ = put(nodes, off, X)
        got = gp.gp_predict(pn, po, dX).cpu().numpy()
        want = oracle.predict32(nodes, off, X)
        np.testing.assert_array_equal(got.view(np.uint32), want.view(np.uint32))


def test_predict_tiny_programs_and_protected_points():
    rows = read_table("tiny_programs.txt")
    nodes, off = pack([parse_prefix(r[0]) for r in rows])
    rng = np.random.default_rng(2)
    X = rng.uniform(-5, 5, size=(2, 1000)).astype(np.float32)
    X[:, :6] = np.array([[0.0, 0.0005, -0.000999, 0.001, 1.5, -2.25],
                         [0.0011, -0.0005, 0.002, -0.001, 0.0, 3.0]], np.float32)
    pn, po, dX, _, _ = put(nodes, off, X)
    got = gp.gp_predict(pn, po, dX).cpu().numpy()
    st, _ = check_points(got, nodes, off, X)
    assert st.ok > 0.6 * st.rows


def test_special_values_through_every_operator():
    """NaN, +-inf, +-0, denormals, huge values and both sides of the
    protection threshold through every operator (alone, with a terminal
    operand on either side and with a stack operand): the GPU gives the FP64
    oracle's class (NaN / +inf / -inf / finite) wherever the FP32 oracle
    agrees with it, and finite values within the per-point bound."""
    sp = np.array([np.nan, np.inf, -np.inf, 0.0, -0.0, 1e-40, -1e-40, 3e38, -3e38, 0.000999,
                   -0.000999, 0.001, -0.001, 0.0011, 1.0, -2.5, 70000.0, 1e30, 88.8, -104.0],
                  np.float32)
    a, b = np.meshgrid(sp, sp)
    X = np.stack([a.ravel(), b.ravel()]).astype(np.float32)
    progs = []
    for name in ("sqrt", "log", "exp", "sin", "cos", "tan", "abs", "neg", "inv", "sq", "cube",
                 "cbrt", "tanh", "atan", "sinh", "cosh"):
        progs.append(parse_prefix(f"{name} x0"))
        progs.append(parse_prefix(f"add {name} x0 {name} x1"))
    for name in ("add", "sub", "mul", "div", "max", "min"):
        progs.append(parse_prefix(f"{name} x0 x1"))
        progs.append(parse_prefix(f"{name} x0 0.5"))
        progs.append(parse_prefix(f"{name} -0.75 x1"))
        progs.append(parse_prefix(f"{name} neg x0 neg x1"))
    nodes, off = pack(progs)
    pn, po, dX, _, _ = put(nodes, off, X)
    got = gp.gp_predict(pn, po, dX).cpu().numpy()
    v64 = oracle.predict64(nodes, off, X)[0]
    v32 = oracle.predict32(nodes, off, X).astype(np.float64)

    def cls(v):
        return np.where(np.isnan(v), 0, np.where(v == np.inf, 1, np.where(v == -np.inf, 2, 3)))

    agree = cls(v64) == cls(v32)
    np.testing.assert_array_equal(cls(got)[agree], cls(v64)[agree])
    assert agree.mean() > 0.9
    st, _ = check_points(got, nodes, off, X)
    assert st.ok > 0.3 * st.rows, st


@pytest.mark.parametrize("n_feat,funcs", [(2, synth.FULL_SET), (1, synth.FULL_SET + ("tan",)),
                                          (7, synth.FULL_SET + ("tan",)), (50, synth.FULL_SET),
                                          (2, synth.EXTENDED_SET), (9, synth.EXTENDED_SET)])
def test_predict_full_function_set(n_feat, funcs):
    nodes, off = synth.ramped_half_and_half(600, 2, 8, funcs, n_feat, seed=40 + n_feat)
    n = 2048 + 61
    X = np.random.default_rng(n_feat).uniform(-5, 5, size=(n_feat, n)).astype(np.float32)
    pn, po, dX, _, _ = put(nodes, off, X)
    got = gp.gp_predict(pn, po, dX).cpu().numpy()
    st, _ = check_points(got, nodes, off, X)
    assert st.ok > 0.5 * st.rows, st


def test_constant_subtrees_fold_to_the_per_row_value():
    """The pre-pass folds every constant-only subtree into one constant,
    computed with the evaluator's own FP32 operations.  Columns 0-2 of X hold
    one value each on every row; replacing each read of such a column by a
    constant of that value makes those subtrees constant-only, and the
    predictions must not change by a single bit (values below the protection
    threshold, on the trig slow path, zero and negative included)."""
    cval = np.array([0.0005, 70000.0, -3.75], np.float32)
    funcs = synth.EXTENDED_SET
    nodes, off = synth.ramped_half_and_half(800, 2, 8, funcs, 6, seed=77)
    n = 1024 + 45
    X = np.random.default_rng(5).uniform(-5, 5, size=(6, n)).astype(np.float32)
    X[:3] = cval[:, None]
    folded = nodes.copy()
    is_const_col = (folded["op"] == synth.OP["var"]) & (folded["feat"] < 3)
    folded["c"][is_const_col] = cval[folded["feat"][is_const_col]]
    folded["op"][is_const_col] = synth.OP["const"]
    folded["feat"][is_const_col] = 0
    assert is_const_col.sum() > 300
    a = gp.gp_predict(*put(nodes, off, X)[:3]).cpu().numpy()
    b = gp.gp_predict(*put(folded, off, X)[:3]).cpu().numpy()
    nan = np.isnan(a)
    np.testing.assert_array_equal(nan, np.isnan(b))
    np.testing.assert_array_equal(a[~nan].view(np.uint32), b[~nan].view(np.uint32))
    # the same through the loop at 8 rows per lane
    a8 = gp.gp_predict_ex(*put(nodes, off, X)[:3], gp.make_opts(rows_per_thread=8)).cpu().numpy()
    np.testing.assert_array_equal(nan, np.isnan(a8))
    np.testing.assert_array_equal(a[~nan].view(np.uint32), a8[~nan].view(np.uint32))
    # and the folded programs still agree with the oracle
    st, _ = check_points(b, folded, off, X)
    assert st.ok > 0.5 * st.rows, st


def _edge_arguments():
    """Arguments at and around every edge of the fast loop's paths: zero,
    subnormals, the protection threshold, the square root's and the
    division's range limits, exp's fast range (87), its overflow and
    underflow ends (89, -110), the trigonometric range (65536), the
    reciprocal's (2^126), huge values, infinities and NaN."""
    v = [0.0, 1e-40, 2.0 ** -101, 2.0 ** -99, 2.0 ** -61, 2.0 ** -59, 0.000999, 0.001, 0.0011,
         0.5, 1.0, 3.25, 86.9, 87.0, 88.0, 88.72, 88.73, 89.0, 100.0, 103.9, 104.0, 109.9,
         110.0, 120.0, 65535.0, 65536.0, 70000.0, 2.0 ** 59, 2.0 ** 61, 2.0 ** 125, 2.0 ** 126,
         2.0 ** 127, 3e38, np.inf]
    v = np.array(v, np.float64)
    return np.concatenate([v, -v, [np.nan]]).astype(np.float32)


@pytest.mark.parametrize("rpt", [4, 8])
def test_fast_loop_matches_the_folded_value_at_edge_arguments(rpt):
    """Every operation the fast loop runs gives, on every edge argument, the
    bits of the C++ function the pre-pass folds constants with (NaN where
    it gives NaN): unary functions f(x0) on the rows against f(c) folded,
    and the division both ways against c1 / c2 folded."""
    V, C = synth.OP["var"], synth.OP["const"]
    e = _edge_arguments()
    n = len(e)
    progs = []
    unary = ("sqrt", "log", "exp", "sin", "cos", "inv", "abs", "neg")
    for f in unary:
        progs.append([(synth.OP[f], 0, 0.0), (V, 0, 0.0)])
        progs += [[(synth.OP[f], 0, 0.0), (C, 0, float(c))] for c in e]
    # div x0 x1 over the grid of edge pairs; the folded c1 / c2 for each
    a, b = np.meshgrid(e, e, indexing="ij")
    X = np.stack([a.ravel(), b.ravel()]).astype(np.float32)
    progs.append([(synth.OP["div"], 0, 0.0), (V, 0, 0.0), (V, 1, 0.0)])
    progs.append([(synth.OP["div"], 0, 0.0), (V, 0, 0.0), (C, 0, 0.75)])
    progs.append([(synth.OP["div"], 0, 0.0), (C, 0, -2.5), (V, 1, 0.0)])
    folded = [[(synth.OP["div"], 0, 0.0), (C, 0, float(x)), (C, 0, float(y))]
              for x, y in zip(a.ravel(), b.ravel())]
    folded += [[(synth.OP["div"], 0, 0.0), (C, 0, float(x)), (C, 0, 0.75)] for x in e]
    folded += [[(synth.OP["div"], 0, 0.0), (C, 0, -2.5), (C, 0, float(y))] for y in e]
    nodes, off = pack(progs + folded)
    pn, po, dX, _, _ = put(nodes, off, X)
    got = gp.gp_predict_ex(pn, po, dX, gp.make_opts(rows_per_thread=rpt)).cpu().numpy()

    def same(x, y, what):
        nan = np.isnan(y)
        np.testing.assert_array_equal(np.isnan(x), nan, err_msg=what)
        np.testing.assert_array_equal(x[~nan].view(np.uint32), y[~nan].view(np.uint32),
                                      err_msg=what)

    # X[0] holds the edge values on rows i * n (the grid's first column)
    rows = np.arange(n) * n
    for k, f in enumerate(unary):
        base = k * (n + 1)
        same(got[base, rows], got[base + 1:base + 1 + n, 0], f)
    d0 = len(unary) * (n + 1)
    fb = len(progs)
    same(got[d0], got[fb:fb + n * n, 0], "div x0 x1")
    same(got[d0 + 1, rows], got[fb + n * n:fb + n * n + n, 0], "div x0 0.75")
    same(got[d0 + 2, :n], got[fb + n * n + n:fb + n * n + 2 * n, 0], "div -2.5 x1")


def _special_rows(X, seed):
    """Overwrite a scattering of rows with values that reach the protected
    branches and the slow paths: zero, both sides of the threshold,
    arguments of exp beyond 87 and of sin/cos beyond 65536, huge, inf, NaN."""
    vals = np.array([0.0, -0.0, 0.0005, -0.0009999, 0.001, 0.0011, 88.5, -100.0, 70000.0,
                     1e30, -1e30, np.inf, -np.inf, np.nan, 1e-40], np.float32)
    rng = np.random.default_rng(seed)
    for f in range(X.shape[0]):
        idx = rng.choice(X.shape[1], size=3 * len(vals), replace=False)
        X[f, idx] = np.tile(vals, 3)
    return X


@pytest.mark.parametrize("n_feat,funcs", [(2, synth.FULL_SET + ("tan",)), (1, synth.FULL_SET),
                                          (9, synth.FULL_SET + ("tan",)),
                                          (2, synth.EXTENDED_SET)])
def test_predictions_do_not_depend_on_rows_per_thread(n_feat, funcs):
    """The fast loop at 8 rows per lane (four packed pairs) gives every row
    the bits of the loop at 4 rows per lane: each row's operations are the
    same whichever way rows are grouped, and a warp that hands a word back
    (trig or exp argument off the fast path) has it done by the same C++
    functions."""
    nodes, off = synth.ramped_half_and_half(900, 2, 8, funcs, n_feat, seed=60 + n_feat)
    n = 4096 + 37
    X = np.random.default_rng(n_feat).uniform(-6, 6, size=(n_feat, n)).astype(np.float32)
    X = _special_rows(X, n_feat)
    pn, po, dX, _, _ = put(nodes, off, X)
    a = gp.gp_predict_ex(pn, po, dX, gp.make_opts(rows_per_thread=4)).cpu().numpy()
    b = gp.gp_predict_ex(pn, po, dX, gp.make_opts(rows_per_thread=8)).cpu().numpy()
    c = gp.gp_predict(pn, po, dX).cpu().numpy()
    for other in (b, c):
        nan = np.isnan(a)
        np.testing.assert_array_equal(nan, np.isnan(other))
        np.testing.assert_array_equal(a[~nan].view(np.uint32), other[~nan].view(np.uint32))
    st, _ = check_points(b, nodes, off, X)
    assert st.ok > 0.5 * st.rows, st


def test_deep_and_long_programs():
    """Programs needing all 20 stack slots (the deep register class), 255
    nodes, single terminals, unary chains."""
    V, Cn = synth.OP["var"], synth.OP["const"]
    progs = []
    for d in (8, 9, 12, 19):  # left spines: stack height d + 1
        progs.append([(synth.OP["sub"], 0, 0.0)] * d + [(V, 0, 0.0)] +
                     [(Cn, 0, float(np.float32(0.125 * (i + 1)))) for i in range(d)])
        progs.append([(synth.OP["div"], 0, 0.0)] * d + [(V, 1, 0.0)] +
                     [(synth.OP["add"], 0, 0.0), (V, 0, 0.0), (V, 1, 0.0)] * d)
    progs.append([(synth.OP["add"], 0, 0.0), (Cn, 0, 1.0)] * 127 + [(V, 0, 0.0)])  # 255 nodes
    progs.append([(synth.OP["sin"], 0, 0.0)] * 254 + [(V, 1, 0.0)])
    progs.append([(V, 1, 0.0)])
    progs.append([(Cn, 0, -3.5)])
    nodes, off = pack(progs)
    for stt, hw in [oracle.validate(nodes[off[i]:off[i + 1]], 2) for i in range(len(progs))]:
        assert stt == oracle.OK and hw <= 20
    X = synth.pagie_data(1000 + 3, 9).X
    pn, po, dX, _, _ = put(nodes, off, X)
    got = gp.gp_predict(pn, po, dX).cpu().numpy()
    check_points(got, nodes, off, X)
    y = synth.pagie_data(1003, 9).y
    fit = gp.gp_evaluate(pn, po, dX, dev(y), metric="mse").cpu().numpy()
    check_fitness(fit, nodes, off, X, y, None, "mse")


def _class_mix(n_feat, seed):
    """Programs for each evaluator class: the usual set with a compiled stack
    of at most 7 (class 0), the extended set with at most 8 (class 2), and
    left spines whose right operands are subtrees, which keep d + 1 values on
    the stack, over both sets: d = 6 and 7 at the edges of classes 0 and 3
    (the usual set at exactly 8) and class 2, deeper ones in class 1."""
    V, Cn = synth.OP["var"], synth.OP["const"]
    usual = synth.unpack(*synth.ramped_half_and_half(150, 2, 6, synth.FULL_SET, n_feat, seed=seed))
    ext = synth.unpack(*synth.ramped_half_and_half(150, 2, 6, synth.EXTENDED_SET, n_feat,
                                                   seed=seed + 1))
    deep = []
    for d in (6, 7, 9, 12, 19):
        deep.append([(synth.OP["max"], 0, 0.0)] * d + [(V, 1 % n_feat, 0.0)] +
                    [(synth.OP["tanh"], 0, 0.0), (V, 0, 0.0)] * d)
        deep.append([(synth.OP["add"], 0, 0.0)] * d + [(V, 1 % n_feat, 0.0)] +
                    [(synth.OP["mul"], 0, 0.0), (V, 0, 0.0), (Cn, 0, 0.5)] * d)
        deep.append([(synth.OP["sub"], 0, 0.0)] * d + [(V, 0, 0.0)] +
                    [(synth.OP["cube"], 0, 0.0), (synth.OP["sin"], 0, 0.0), (V, 1 % n_feat, 0.0)] * d)
    return [usual, ext, deep]


@pytest.mark.parametrize("n_feat", [2, 9])
@pytest.mark.parametrize("metric", ["rmse", "pearson"])
def test_fitness_in_every_program_class(n_feat, metric):
    """One population, interleaved, whose programs fall into all four
    evaluator classes (6-slot stack, 7-slot stack without and with the
    extended functions, 19-slot stack): at 4 and at 8 rows per thread for
    the common class, every fitness matches the oracle's, and equals, bit for
    bit, the fitness of the same programs evaluated one group at a time with
    the same row chunks (each class reads its own span of the program
    order)."""
    groups = _class_mix(n_feat, 300 + n_feat)
    n = 2 * 4096 + 77
    rng = np.random.default_rng(n_feat)
    X = rng.uniform(-3, 3, size=(n_feat, n)).astype(np.float32)
    y = (X[0] * np.float32(0.75) + np.tanh(X[1 % n_feat])).astype(np.float32)
    w = _weights(n, 4)
    progs, where = [], []
    for g, grp in enumerate(groups):
        for i, pr in enumerate(grp):
            progs.append(pr)
            where.append((g, i))
    perm = np.random.default_rng(1).permutation(len(progs))
    progs = [progs[i] for i in perm]
    where = [where[i] for i in perm]
    nodes, off = pack(progs)
    pn, po, dX, dy, dw = put(nodes, off, X, y, w)
    for rpt in (4, 8):
        opts = gp.make_opts(rows_per_thread=rpt, chunk_rows=2048)
        fit = gp.gp_evaluate_ex(pn, po, dX, dy, dw, metric=metric, opts=opts).cpu().numpy()
        if metric == "pearson":
            st, _ = check_pearson(fit, nodes, off, X, y, w)
        else:
            st, _ = check_fitness(fit, nodes, off, X, y, w, metric)
        assert st.flagged < 0.3 * st.programs, st
        for g, grp in enumerate(groups):
            gn, go = pack(grp)
            gpn, gpo = gp.nodes_to_device(gn), dev(go.astype(np.int32))
            alone = gp.gp_evaluate_ex(gpn, gpo, dX, dy, dw, metric=metric,
                                      opts=opts).cpu().numpy()
            mixed = np.array([fit[k] for k in range(len(progs)) if where[k][0] == g])
            idx = [where[k][1] for k in range(len(progs)) if where[k][0] == g]
            np.testing.assert_array_equal(mixed.view(np.uint32), alone[idx].view(np.uint32))


# --------------------------------------------------------------------------
# fitness
# --------------------------------------------------------------------------
def test_fitness_pagie_small_full():
    """Pagie-1, N=4096, P=512, {add,sub,mul,div}, MSE: every program."""
    wl = synth.workload("pagie_small")
    d = wl.data
    pn, po, dX, dy, _ = put(wl.nodes, wl.offsets, d.X, d.y)
    fit = gp.gp_evaluate(pn, po, dX, dy, metric="mse").cpu().numpy()
    stats, f64 = check_fitness(fit, wl.nodes, wl.offsets, d.X, d.y, None, "mse")
    assert stats.strict > 0.8 * stats.programs, stats
    # the GPU values are bit-exact to the oracle's FP32 mode here, so its
    # fitness equals the FP64 reduction of those values up to summation
    p32 = oracle.predict32(wl.nodes, wl.offsets, d.X).astype(np.float64)
    with np.errstate(all="ignore"):
        ref = np.mean((p32 - d.y.astype(np.float64)) ** 2, axis=1)
        fin = np.isfinite(ref)
        np.testing.assert_allclose(fit[fin], ref[fin], rtol=2e-6)


@pytest.mark.parametrize("metric", ["mae", "mse", "rmse", "logloss"])
@pytest.mark.parametrize("weighted", [False, True])
def test_fitness_metrics_ragged_many_chunks(metric, weighted):
    n = 4096 + 37
    if metric == "logloss":
        d = synth.classification_data(n, 7, n_feat=5)
        funcs = synth.FULL_SET
    else:
        d = synth.pagie_data(n, 8)
        funcs = synth.FULL_SET + ("tan",)
    w = _weights(n, 3) if weighted else (d.w if metric == "logloss" else None)
    nodes, off = synth.ramped_half_and_half(256, 2, 7, funcs, d.n_feat, seed=60)
    pn, po, dX, dy, dw = put(nodes, off, d.X, d.y, w)
    for rpt in (4, 8):
        opts = gp.make_opts(rows_per_thread=rpt, chunk_rows=256)
        fit = gp.gp_evaluate_ex(pn, po, dX, dy, dw, metric=metric, opts=opts).cpu().numpy()
        stats, _ = check_fitness(fit, nodes, off, d.X, d.y, w, metric)
        assert stats.strict > 0.5 * stats.programs, stats


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("n_feat", [2, 9])
def test_pearson_fitness(weighted, n_feat):
    """Weighted Pearson fitness |r| over several row chunks and a ragged
    tail: programs from the full set plus exact cases (an affine image of y
    scores 1, constants score 0), both feature modes, every rows-per-thread
    instance."""
    n = 3 * 4096 + 123
    rng = np.random.default_rng(90 + n_feat)
    X = rng.uniform(-4, 4, size=(n_feat, n)).astype(np.float32)
    y = (X[0] * np.float32(0.5) + np.sin(X[1]).astype(np.float32)).astype(np.float32)
    w = _weights(n, 11) if weighted else None
    nodes, off = synth.ramped_half_and_half(300, 2, 7, synth.FULL_SET + ("tan",), n_feat,
                                            seed=91 + n_feat)
    extra = [
        [(synth.OP["const"], 0, 2.0)],
        [(synth.OP["sin"], 0, 0.0), (synth.OP["const"], 0, 0.3)],
        [(synth.OP["var"], 0, 0.0)],
        [(synth.OP["add"], 0, 0.0), (synth.OP["mul"], 0, 0.0), (synth.OP["const"], 0, 0.5),
         (synth.OP["var"], 0, 0.0), (synth.OP["sin"], 0, 0.0), (synth.OP["var"], 1, 0.0)],
        [(synth.OP["neg"], 0, 0.0), (synth.OP["add"], 0, 0.0), (synth.OP["mul"], 0, 0.0),
         (synth.OP["const"], 0, 0.5), (synth.OP["var"], 0, 0.0), (synth.OP["sin"], 0, 0.0),
         (synth.OP["var"], 1, 0.0)],
    ]
    # random programs barely correlate with y (median |r| ~ 0.01), so most
    # can only be held to their propagated bound; programs close to the
    # target's form, c1 x0 + c2 sin(x1) + c3 cos(x0), correlate well and
    # must meet the 1e-4 tolerance
    crng = np.random.default_rng(7)
    close = []
    for _ in range(60):
        c1, c2, c3 = (float(np.float32(v)) for v in crng.uniform(-2, 2, 3))
        close.append([(synth.OP["add"], 0, 0.0), (synth.OP["add"], 0, 0.0),
                      (synth.OP["mul"], 0, 0.0), (synth.OP["const"], 0, c1), (synth.OP["var"], 0, 0.0),
                      (synth.OP["mul"], 0, 0.0), (synth.OP["const"], 0, c2),
                      (synth.OP["sin"], 0, 0.0), (synth.OP["var"], 1, 0.0),
                      (synth.OP["mul"], 0, 0.0), (synth.OP["const"], 0, c3),
                      (synth.OP["cos"], 0, 0.0), (synth.OP["var"], 0, 0.0)])
    nodes, off = pack(synth.unpack(nodes, off) + close + extra)
    n_close = len(close) + len(extra)
    pn, po, dX, dy, dw = put(nodes, off, X, y, w)
    for rpt in (4, 8, 16):
        opts = gp.make_opts(rows_per_thread=rpt, chunk_rows=1024)
        fit = gp.gp_evaluate_ex(pn, po, dX, dy, dw, metric="pearson", opts=opts).cpu().numpy()
        st, f64 = check_pearson(fit, nodes, off, X, y, w)
        assert st.flagged < 0.3 * st.programs, st
        st_close, _ = check_pearson(fit[-n_close:], *pack(close + extra), X, y, w)
        assert st_close.strict >= 0.8 * len(close), st_close
        assert fit[-5] == 0.0 and fit[-4] == 0.0
        assert fit[-2] == pytest.approx(1.0, abs=2e-6) and fit[-1] == pytest.approx(1.0, abs=2e-6)
    # the default entry point and the host entry point agree with the above
    fit_d = gp.gp_evaluate(pn, po, dX, dy, dw, metric="pearson").cpu().numpy()
    check_pearson(fit_d, nodes, off, X, y, w)
    fit_h = gp.gp_evaluate_host(nodes, off, X, y, w, metric="pearson")
    np.testing.assert_array_equal(np.isnan(fit_h), np.isnan(fit_d))
    # selection on |r| (greater is better) is the oracle's, bit for bit
    win = gp.gp_tournament_ex(torch.from_numpy(fit_d).cuda(), 400, 20, 5,
                              greater_is_better=True).cpu().numpy()
    np.testing.assert_array_equal(win, oracle.tournament(fit_d, 400, 20, 5, greater_is_better=True))


@pytest.mark.parametrize("n,weighted", [(3 * 2048 + 77, False), (40_000, True), (1000, True)])
def test_spearman_fitness(n, weighted):
    """Spearman |r_s| through device ranking: equal (1e-9) to the oracle's
    Spearman of the evaluator's own predictions (the device sort, tie ranks
    and moment sums against their definition), equal to the oracle's
    Spearman of the oracle's FP32 predictions for the IEEE operators (whose
    values are bit-equal), and close to the FP64 oracle otherwise (library
    functions a few ulp apart can break or make ties, and ranks are
    discontinuous); ties in predictions and targets, constant and NaN
    programs, ragged tiles."""
    rng = np.random.default_rng(n)
    X = rng.uniform(-3, 3, size=(3, n)).astype(np.float32)
    X[2] = np.round(X[2])  # a feature with many ties
    y = (X[0] + np.sin(X[1])).astype(np.float32)
    y[: n // 10] = np.round(y[: n // 10])  # ties in the target
    w = _weights(n, 12) if weighted else None
    ieee = synth.ramped_half_and_half(200, 2, 6, ("add", "sub", "mul", "div", "sqrt", "abs", "neg", "inv"),
                                      3, seed=41)
    libm = synth.ramped_half_and_half(200, 2, 6, synth.FULL_SET + ("tan",), 3, seed=42)
    extra = [[(synth.OP["const"], 0, 1.5)],                                   # constant
             [(synth.OP["var"], 2, 0.0)],                                     # tied feature
             [(synth.OP["log"], 0, 0.0), (synth.OP["const"], 0, 0.0)],        # protected: 0
             [(synth.OP["sqrt"], 0, 0.0), (synth.OP["exp"], 0, 0.0), (synth.OP["exp"], 0, 0.0),
              (synth.OP["exp"], 0, 0.0), (synth.OP["var"], 0, 0.0)]]          # inf for large x0
    progs = synth.unpack(*ieee) + synth.unpack(*libm) + extra
    nodes, off = pack(progs)
    pn, po, dX, dy, dw = put(nodes, off, X, y, w)
    fit64 = torch.empty(len(progs), dtype=torch.float64, device="cuda")
    gp.gp_evaluate_ex(pn, po, dX, dy, dw, metric="spearman", out64=fit64)
    fit = fit64.cpu().numpy()
    gpred = gp.gp_predict(pn, po, dX).cpu().numpy().astype(np.float64)
    p32 = oracle.predict32(nodes, off, X).astype(np.float64)
    f64, st = oracle.fitness(nodes, off, X, y, w, "spearman")
    n_ieee = len(ieee[1]) - 1
    stable = 0
    for i in range(len(progs)):
        own = oracle.spearman_of(gpred[i], y, w)
        if np.isnan(own):
            assert np.isnan(fit[i]), i
            continue
        assert abs(fit[i] - own) <= 1e-9 * max(abs(own), 1e-3), (i, fit[i], own)
        if i < n_ieee:
            ref32 = oracle.spearman_of(p32[i], y, w)
            assert abs(fit[i] - ref32) <= 1e-9 * max(abs(ref32), 1e-3), (i, fit[i], ref32)
        # against the FP64 oracle where the oracle itself shows the program's
        # ranks insensitive to FP32 rounding (its FP32 and FP64 values give
        # the same coefficient); ranks are discontinuous, so elsewhere FP32
        # may tie or order rows differently and the difference is not bounded
        # (for the library functions the device values may still sit a few
        # ulp from the oracle's and swap a few neighbours: one swap of
        # adjacent ranks moves r_s by at most 12 / n^2; four are allowed)
        if np.isfinite(f64[i]) and np.all(np.isfinite(p32[i])):
            if abs(oracle.spearman_of(p32[i], y, w) - f64[i]) <= 1e-9:
                tol = 1e-6 if i < n_ieee else max(1e-6, 48.0 / n ** 2)
                assert abs(fit[i] - f64[i]) <= tol, (i, fit[i], f64[i])
                stable += 1
    assert stable > 150
    assert fit[-4] == 0.0
    assert fit[-2] == 0.0 or np.isnan(fit[-2])


@pytest.mark.parametrize("n_rows,n_progs", [(1 << 21, 300), (1 << 20, 4096)])
def test_spearman_over_several_batches(n_rows, n_progs):
    """The ranks of at most 2 GB of predictions are sorted at a time (42
    programs per batch at 2M rows, 85 at 1M: the second case is the
    Spearman configuration bench.py times, 49 batches); sampled programs
    from every batch equal the oracle's Spearman of the device's FP32
    predictions."""
    wl = synth.workload("pagie_large", n_rows=n_rows, n_progs=n_progs)
    d = wl.data
    pn, po, dX, dy, _ = put(wl.nodes, wl.offsets, d.X, d.y)
    fit64 = torch.empty(n_progs, dtype=torch.float64, device="cuda")
    gp.gp_evaluate_ex(pn, po, dX, dy, metric="spearman", out64=fit64)
    fit = fit64.cpu().numpy()
    idx = np.arange(3, n_progs, max(19, n_progs // 20))
    sn, so = _subset(wl.nodes, wl.offsets, idx)
    gpred = gp.gp_predict(gp.nodes_to_device(sn), dev(so), dX).cpu().numpy().astype(np.float64)
    checked = 0
    for k, i in enumerate(idx):
        ref = oracle.spearman_of(gpred[k], d.y)
        if np.isnan(ref):
            assert np.isnan(fit[i])
            continue
        assert abs(fit[i] - ref) <= 1e-9 * max(ref, 1e-3), (i, fit[i], ref)
        checked += 1
    assert checked >= 10


def test_pearson_rejected_where_unsupported():
    d = synth.pagie_data(1024, 3)
    nodes, off = synth.ramped_half_and_half(8, 2, 4, synth.FULL_SET, 2, seed=3)
    pn, po, dX, dy, _ = put(nodes, off, d.X, d.y)
    with pytest.raises(gp.GPError):
        gp.gp_evaluate_plain(pn, po, dX, dy, metric="pearson")
    with pytest.raises(gp.GPError):
        gp.gp_const_grad(pn, po, dX, dy, metric="pearson")
    for m in ("spearman",):
        with pytest.raises(gp.GPError):
            gp.gp_evaluate_plain(pn, po, dX, dy, metric=m)
        with pytest.raises(gp.GPError):
            gp.gp_evaluate_static(pn, po, dX, dy, metric=m)
        with pytest.raises(gp.GPError):
            gp.gp_autotune(pn, po, dX, dy, metric=m)


def test_length_bucket_split():
    """The common class split at a compiled-length edge into a long and a
    short launch: with the same rows per thread every fitness is the
    unsplit one, bit for bit (the bucket a program lands in does not change
    its reduction); with 8 rows per thread for the long bucket it still
    matches the oracle."""
    n = 3 * 16384 + 77
    d = synth.pagie_data(n, 21)
    nodes, off = synth.ramped_half_and_half(700, 2, 9, synth.FULL_SET, 2, seed=22)
    pn, po, dX, dy, _ = put(nodes, off, d.X, d.y)
    base = gp.gp_evaluate_ex(pn, po, dX, dy, metric="rmse",
                             opts=gp.make_opts(rows_per_thread=4, chunk_rows=4096,
                                               long_edge=-1)).cpu().numpy()
    for edge in (1, 12, 24, 255):
        split = gp.gp_evaluate_ex(pn, po, dX, dy, metric="rmse",
                                  opts=gp.make_opts(rows_per_thread=4, chunk_rows=4096,
                                                    long_edge=edge, long_rows_per_thread=4,
                                                    long_blocks_per_sm=2)).cpu().numpy()
        nan = np.isnan(base)
        np.testing.assert_array_equal(nan, np.isnan(split))
        np.testing.assert_array_equal(base[~nan].view(np.uint32), split[~nan].view(np.uint32))
    mixed = gp.gp_evaluate_ex(pn, po, dX, dy, metric="rmse",
                              opts=gp.make_opts(rows_per_thread=4, chunk_rows=4096, long_edge=16,
                                                long_rows_per_thread=8)).cpu().numpy()
    st, _ = check_fitness(mixed, nodes, off, d.X, d.y, None, "rmse")
    assert st.strict > 0.5 * st.programs, st
    with pytest.raises(gp.GPError):
        gp.gp_evaluate_ex(pn, po, dX, dy, opts=gp.make_opts(long_edge=300))
    with pytest.raises(gp.GPError):
        gp.gp_evaluate_ex(pn, po, dX, dy, opts=gp.make_opts(long_edge=8, long_rows_per_thread=5))


def test_autotune_choice_is_used_and_correct():
    """gp_autotune's choice is recorded for the shape: a later call with
    zero tunables uses it (fitness bit-equal to gp_evaluate_ex with the
    returned opts), and that fitness matches the oracle."""
    wl = synth.workload("pagie_large", n_rows=1 << 18, n_progs=512)
    d = wl.data
    pn, po, dX, dy, _ = put(wl.nodes, wl.offsets, d.X, d.y)
    best = gp.gp_autotune(pn, po, dX, dy, metric=wl.metric)
    assert best.rows_per_thread in (4, 8) and best.chunk_rows % 256 == 0
    assert best.long_edge == -1 or 1 <= best.long_edge <= 255
    used = gp.gp_resolve_opts(512, d.n_rows, d.n_feat)
    assert (used.rows_per_thread, used.chunk_rows, used.long_edge) == \
        (best.rows_per_thread, best.chunk_rows, best.long_edge)
    a = gp.gp_evaluate(pn, po, dX, dy, metric=wl.metric).cpu().numpy()
    b = gp.gp_evaluate_ex(pn, po, dX, dy, metric=wl.metric, opts=best).cpu().numpy()
    nan = np.isnan(a)
    np.testing.assert_array_equal(nan, np.isnan(b))
    np.testing.assert_array_equal(a[~nan].view(np.uint32), b[~nan].view(np.uint32))
    idx = _sample(wl.offsets, 24, 3)
    sn, so = _subset(wl.nodes, wl.offsets, idx)
    st, _ = check_fitness(a[idx], sn, so, d.X, d.y, None, wl.metric)
    assert st.strict >= 8, st


def test_plain_evaluator_matches_oracle_and_batched():
    wl = synth.workload("pagie_small")
    d = wl.data
    w = _weights(d.n_rows, 4)
    pn, po, dX, dy, dw = put(wl.nodes, wl.offsets, d.X, d.y, w)
    plain = gp.gp_evaluate_plain(pn, po, dX, dy, dw, metric="rmse").cpu().numpy()
    batched = gp.gp_evaluate(pn, po, dX, dy, dw, metric="rmse").cpu().numpy()
    check_fitness(plain, wl.nodes, wl.offsets, d.X, d.y, w, "rmse")
    fin = np.isfinite(batched)
    np.testing.assert_array_equal(np.isfinite(plain), fin)
    np.testing.assert_allclose(plain[fin], batched[fin], rtol=2e-6)


def test_fitness_is_deterministic_and_accumulators_agree():
    wl = synth.workload("pagie_large", n_rows=1 << 16, n_progs=512)
    d = wl.data
    pn, po, dX, dy, _ = put(wl.nodes, wl.offsets, d.X, d.y)
    a = gp.gp_evaluate(pn, po, dX, dy, metric="rmse").cpu().numpy()
    b = gp.gp_evaluate(pn, po, dX, dy, metric="rmse").cpu().numpy()
    np.testing.assert_array_equal(a.view(np.uint32), b.view(np.uint32))
    o64 = gp.make_opts(rows_per_thread=8, chunk_rows=1024, accum="fp64")
    o32 = gp.make_opts(rows_per_thread=8, chunk_rows=1024, accum="kahan32")
    f64 = gp.gp_evaluate_ex(pn, po, dX, dy, metric="rmse", opts=o64).cpu().numpy()
    f32 = gp.gp_evaluate_ex(pn, po, dX, dy, metric="rmse", opts=o32).cpu().numpy()
    fin = np.isfinite(f64)
    np.testing.assert_allclose(f32[fin], f64[fin], rtol=1e-6)
    np.testing.assert_allclose(a[fin], f64[fin], rtol=5e-6)
    stats, _ = check_fitness(a, wl.nodes, wl.offsets, d.X, d.y, None, "rmse")
    assert stats.strict > 0.5 * stats.programs


def test_invalid_programs_are_flagged_not_trapped():
    good = parse_prefix("add x0 x1")
    V, A = synth.OP["var"], synth.OP["add"]
    progs = [good, [(A, 0, 0.0), (V, 0, 0.0)], good, [(V, 5, 0.0)], [(99, 0, 0.0)],
             [(V, 0, 0.0), (V, 1, 0.0)], [(A, 0, 0.0)] * 21 + [(V, 0, 0.0)] * 22, good]
    nodes, off = pack(progs)
    d = synth.pagie_data(300, 1)
    pn, po, dX, dy, _ = put(nodes, off, d.X, d.y)
    gp.gp_last_device_status()  # clear
    st = torch.empty(len(progs), dtype=torch.int32, device="cuda")
    fit = gp.gp_evaluate_ex(pn, po, dX, dy, metric="mae", out_status=st).cpu().numpy()
    flags = gp.gp_last_device_status()
    assert flags & gp.DEV_BAD_PROGRAM
    bad = np.array([0, 1, 0, 1, 1, 1, 1, 0], bool)
    assert np.all(np.isnan(fit[bad])) and np.all(np.isfinite(fit[~bad]))
    want = [oracle.validate(nodes[off[i]:off[i + 1]], 2)[0] for i in range(len(progs))]
    np.testing.assert_array_equal(st.cpu().numpy(), np.array(want))
    pred = gp.gp_predict(pn, po, dX).cpu().numpy()
    assert np.all(np.isnan(pred[bad])) and np.all(np.isfinite(pred[~bad]))
    assert gp.gp_last_device_status() & gp.DEV_BAD_PROGRAM
    assert gp.gp_last_device_status() == 0


def test_argument_errors_return_codes():
    d = synth.pagie_data(64, 1)
    nodes, off = pack([parse_prefix("add x0 x1")])
    pn, po, dX, dy, _ = put(nodes, off, d.X, d.y)
    with pytest.raises(gp.GPError) as e:
        gp.gp_evaluate(pn, po, dX, dy, metric=7)
    assert e.value.code == -1
    with pytest.raises(gp.GPError):
        gp.gp_evaluate_ex(pn, po, dX, dy, opts=gp.make_opts(rows_per_thread=3))
    with pytest.raises(gp.GPError) as e:
        gp.gp_evaluate_host(pack([[(synth.OP["add"], 0, 0.0)]])[0], np.array([0, 1], np.int32),
                            d.X, d.y)
    assert e.value.code == -2
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(gp.GPError) as e:
        gp.gp_evaluate_ex(pn, po, dX, dy, ws=small)
    assert e.value.code == -7


def test_edge_sizes():
    nodes, off = synth.ramped_half_and_half(40, 1, 4, synth.FULL_SET, 2, seed=3)
    for n in (1, 2, 3, 4, 5, 127, 129, 1023):
        d = synth.pagie_data(n, n)
        pn, po, dX, dy, _ = put(nodes, off, d.X, d.y)
        fit = gp.gp_evaluate(pn, po, dX, dy, metric="mae").cpu().numpy()
        check_fitness(fit, nodes, off, d.X, d.y, None, "mae")
        pred = gp.gp_predict(pn, po, dX).cpu().numpy()
        check_points(pred, nodes, off, d.X)


def test_host_entry_point_matches_device_entry_point():
    wl = synth.workload("binary", n_rows=8192 + 5, n_progs=128)
    d = wl.data
    host = gp.gp_evaluate_host(wl.nodes, wl.offsets, d.X, d.y, d.w, metric="logloss")
    pn, po, dX, dy, dw = put(wl.nodes, wl.offsets, d.X, d.y, d.w)
    devf = gp.gp_evaluate(pn, po, dX, dy, dw, metric="logloss").cpu().numpy()
    np.testing.assert_array_equal(host.view(np.uint32), devf.view(np.uint32))
    check_fitness(host, wl.nodes, wl.offsets, d.X, d.y, d.w, "logloss")


def test_graph_capture_replays_the_generation():
    wl = synth.workload("pagie_large", n_rows=1 << 15, n_progs=256)
    d = wl.data
    pn, po, dX, dy, _ = put(wl.nodes, wl.offsets, d.X, d.y)
    opts = gp.make_opts(rows_per_thread=4, chunk_rows=2048)
    ws = torch.empty(gp.gp_workspace_size(256, d.n_rows, 2, opts), dtype=torch.uint8, device="cuda")
    fit = torch.empty(256, dtype=torch.float32, device="cuda")
    win = torch.empty(256, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        gp.gp_evaluate_ex(pn, po, dX, dy, metric="rmse", opts=opts, out=fit, ws=ws)
        gp.gp_tournament_ex(fit, 256, 20, 42, out=win)
    s.synchronize()
    eager_fit, eager_win = fit.clone(), win.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        gp.gp_evaluate_ex(pn, po, dX, dy, metric="rmse", opts=opts, out=fit, ws=ws)
        gp.gp_tournament_ex(fit, 256, 20, 42, out=win)
    fit.zero_()
    win.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(fit.view(torch.int32), eager_fit.view(torch.int32))
    assert torch.equal(win, eager_win)


# --------------------------------------------------------------------------
# tournament selection: bit-exact
# --------------------------------------------------------------------------
def test_tournament_bit_exact():
    rng = np.random.default_rng(0)
    for P, T, k in ((512, 512, 20), (1000, 1700, 10), (7, 50, 1), (4096, 7000, 33)):
        f = rng.normal(size=P).astype(np.float32)
        f[rng.random(P) < 0.05] = np.nan
        f[rng.random(P) < 0.05] = np.inf
        f[: P // 4] = np.round(f[: P // 4], 1)  # many ties
        lens = rng.integers(1, 256, P)
        off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
        for pars, greater, seed, offset in ((0.0, False, 42, 0), (0.01, False, 7, 3),
                                            (0.003, True, 2 ** 40 + 5, 2 ** 33)):
            got = gp.gp_tournament_ex(dev(f), T, k, seed, offsets=dev(off), parsimony=pars,
                                      greater_is_better=greater, offset=offset).cpu().numpy()
            want = oracle.tournament(f, T, k, seed, lengths=np.diff(off), parsimony=pars,
                                     greater_is_better=greater, offset=offset)
            np.testing.assert_array_equal(got, want)
    f = rng.normal(size=300).astype(np.float32)
    got = gp.gp_tournament(dev(f), 20, 42).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.tournament(f, 300, 20, 42))


# --------------------------------------------------------------------------
# constant gradients and Adam
# --------------------------------------------------------------------------
@pytest.mark.parametrize("metric,funcs", [("mse", synth.FULL_SET), ("rmse", synth.FULL_SET),
                                          ("mae", synth.FULL_SET), ("logloss", synth.FULL_SET),
                                          ("mse", synth.EXTENDED_SET)])
def test_const_grad_matches_oracle_reverse_mode(metric, funcs):
    n = 2048 + 19
    if metric == "logloss":
        d = synth.classification_data(n, 11, n_feat=4)
    else:
        d = synth.pagie_data(n, 12)
    nodes, off = synth.ramped_half_and_half(200, 2, 6, funcs, d.n_feat, seed=70,
                                            max_consts=16)
    pn, po, dX, dy, dw = put(nodes, off, d.X, d.y, d.w)
    g, f = gp.gp_const_grad(pn, po, dX, dy, dw, metric=metric)
    g, f = g.cpu().numpy().astype(np.float64), f.cpu().numpy()
    g64, f64, gabs = oracle.const_grad(nodes, off, d.X, d.y, d.w, metric, with_abs=True)
    g32, _ = oracle.const_grad32(nodes, off, d.X, d.y, d.w, metric)
    v, e, fl = oracle.predict_bound(nodes, off, d.X, ulps_fn=4.0)
    fbatch = gp.gp_evaluate(pn, po, dX, dy, dw, metric=metric).cpu().numpy()
    # the gradient kernel's fitness and the evaluator's use different FP32
    # function implementations (CUDA's sinf / cosf against the evaluator's
    # own) and summation orders: they agree where every row value is
    # certified to 1e-6 by the error bound
    with np.errstate(invalid="ignore"):
        cert = ~(fl != 0).any(axis=1) & ((e <= 1e-6 * np.abs(v)) | (e <= 1e-30)).all(axis=1)
    cert &= np.isfinite(fbatch)
    assert cert.sum() > 0.2 * len(cert)
    np.testing.assert_allclose(f[cert], fbatch[cert], rtol=2e-5)
    extra = _mae_flip_tol(nodes, off, d, metric)
    strict, cond = _grad_check(g, g64, g32, gabs, fl, extra, e, v)
    assert strict > 0.4 * len(g64), (strict, cond)
    nconst = np.array([oracle.count_consts(nodes[off[i]:off[i + 1]]) for i in range(len(off) - 1)])
    for i, k in enumerate(nconst):
        assert np.all(g[i, k:] == 0)


def _mae_flip_tol(nodes, off, d, metric):
    """MAE's gradient uses sign(p - y): on rows where |p - y| is within
    twice the FP32 value bound the sign may differ between FP32 and FP64,
    which moves the gradient by up to twice those rows' absolute
    contributions.  Returns that amount per (program, constant)."""
    P = len(off) - 1
    if metric != "mae":
        return np.zeros((P, 16))
    v, e, _ = oracle.predict_bound(nodes, off, d.X, ulps_fn=4.0)
    w = np.ones(d.n_rows, np.float32) if d.w is None else d.w
    out = np.zeros((P, 16))
    for p in range(P):
        risk = np.abs(v[p] - d.y) <= 2 * e[p] + 1e-30
        if not risk.any():
            continue
        wr = np.where(risk, w, 0).astype(np.float32)
        sn, so = pack([synth.unpack(nodes, off)[p]])
        _, _, ga = oracle.const_grad(sn, so, d.X, d.y, wr, "mae", with_abs=True)
        out[p] = 2 * ga[0] * wr.sum() / w.sum()
    return out


def _grad_check(g, g64, g32, gabs, fl, extra=None, e=None, v=None):
    """Gradient tolerance.  A gradient inherits the conditioning of the row
    values it is built from, so only programs whose every row value is
    certified to 1e-5 by the FP32 error bound (and has no flagged row) are
    compared: strictly, at 1e-4 of the gradient's scale (the sum of
    absolute per-row contributions), where FP32 rounding alone moves the
    oracle's own FP32 adjoint by less than a quarter of that; otherwise
    within ten times that FP32 deviation.  Other programs are counted."""
    usable = ~(fl != 0).any(axis=1) & np.isfinite(g64).all(axis=1) & np.isfinite(g32).all(axis=1)
    if e is not None:
        with np.errstate(invalid="ignore"):
            usable &= ((e <= 1e-5 * np.abs(v)) | (e <= 1e-30)).all(axis=1)
    with np.errstate(invalid="ignore"):
        tol = 1e-4 * np.maximum(gabs, 1e-3 * np.abs(g64).max(axis=1, keepdims=True)) + 1e-7
        if extra is not None:
            tol = tol + extra
        dev32 = np.abs(g32 - g64)
        well = usable & (dev32 <= 0.25 * tol).all(axis=1)
        ill = usable & ~well
        err = np.abs(g - g64)
    bad = well[:, None] & ~(err <= tol)
    assert not bad.any(), (np.argwhere(bad)[:5], g[bad][:5], g64[bad][:5])
    bad2 = ill[:, None] & ~(err <= 10.0 * dev32 + tol)
    assert not bad2.any(), (np.argwhere(bad2)[:5], g[bad2][:5], g64[bad2][:5], g32[bad2][:5])
    return int(well.sum()), int(ill.sum())


def test_adam_steps_match_oracle():
    d = synth.pagie_data(1024, 5)
    nodes, off = synth.ramped_half_and_half(64, 2, 5, synth.FULL_SET, 2, seed=71, max_consts=16)
    pn, po, dX, dy, _ = put(nodes, off, d.X, d.y)
    m = torch.zeros((64, 16), device="cuda")
    v = torch.zeros((64, 16), device="cuda")
    theta = nodes["c"].astype(np.float64)
    om = np.zeros((64, 16))
    ov = np.zeros((64, 16))
    for step in range(1, 6):
        g, _ = gp.gp_const_grad(pn, po, dX, dy, metric="mse")
        gh = g.cpu().numpy().astype(np.float64)
        gp.gp_adam_step(pn, po, g, m, v, step, lr=1e-2)
        after = gp.nodes_from_device(pn)
        # oracle Adam on the same gradients, parameter per constant slot
        cur = nodes.copy()
        cur["c"] = np.float32(theta)
        for p in range(64):
            idx = np.arange(off[p], off[p + 1])
            kidx = idx[nodes["op"][idx] == synth.OP["const"]]
            if len(kidx) == 0:
                continue
            # a slot whose gradient is not finite keeps its constant and state
            fin = np.isfinite(gh[p, :len(kidx)])
            kf = kidx[fin]
            th = theta[kf].copy()
            mm = om[p, :len(kidx)][fin].copy()
            vv = ov[p, :len(kidx)][fin].copy()
            oracle.adam(th, gh[p, :len(kidx)][fin], mm, vv, step, lr=1e-2)
            om[p, np.flatnonzero(fin)] = mm
            ov[p, np.flatnonzero(fin)] = vv
            theta[kf] = th
            np.testing.assert_allclose(after["c"][kf], th, rtol=2e-6, atol=2e-7)
            np.testing.assert_array_equal(after["c"][kidx[~fin]], cur["c"][kidx[~fin]])
        theta = after["c"].astype(np.float64)
    assert np.array_equal(after["op"], nodes["op"])


def test_constants_as_a_differentiable_tensor():
    """gp_get_consts / gp_set_consts move the constants between the nodes and
    a dense [P, 16] tensor (prefix order, bit for bit), and the autograd
    wrapper returns gp_const_grad's fitness and gradient for that tensor."""
    d = synth.pagie_data(4096 + 19, 8)
    nodes, off = synth.ramped_half_and_half(64, 2, 6, synth.FULL_SET, 2, seed=73, max_consts=16)
    pn, po, dX, dy, _ = put(nodes, off, d.X, d.y)
    c = gp.gp_get_consts(pn, po).cpu().numpy()
    want = np.zeros((64, 16), np.float32)
    for p in range(64):
        seg = nodes[off[p]:off[p + 1]]
        cs = seg["c"][seg["op"] == synth.OP["const"]][:16]
        want[p, :len(cs)] = cs
    np.testing.assert_array_equal(c.view(np.uint32), want.view(np.uint32))

    theta = torch.from_numpy(want * np.float32(1.5) - np.float32(0.25)).cuda().requires_grad_(True)
    fit = gp.fitness_of_constants(theta, pn, po, dX, dy, None, "mse")
    back = gp.gp_get_consts(pn, po).cpu().numpy()
    counts = np.array([min(16, int((nodes[off[p]:off[p + 1]]["op"] == synth.OP["const"]).sum()))
                       for p in range(64)])
    live = np.arange(16)[None, :] < counts[:, None]
    np.testing.assert_array_equal(back[live], theta.detach().cpu().numpy()[live])
    g_ref, f_ref = gp.gp_const_grad(pn, po, dX, dy, metric="mse")
    # bit for bit, NaN where the program's value leaves the float range
    torch.testing.assert_close(fit.detach(), f_ref, rtol=0, atol=0, equal_nan=True)
    wts = torch.rand(64, device="cuda")
    (fit * wts).sum().backward()
    torch.testing.assert_close(theta.grad, g_ref * wts.unsqueeze(1), rtol=0, atol=0,
                               equal_nan=True)
    fin = torch.isfinite(f_ref).cpu().numpy()
    assert fin.sum() > 40
    assert torch.all(theta.grad.cpu()[torch.from_numpy(~live & fin[:, None])] == 0)
    # the fitness of the rewritten programs agrees with the oracle
    moved = gp.nodes_from_device(pn)
    check_fitness(fit.detach().cpu().numpy(), moved, off, d.X, d.y, None, "mse")


# --------------------------------------------------------------------------
# full-size workloads in the benchmark's launch configuration (sampled)
# --------------------------------------------------------------------------
def _sample(off, k, seed):
    P = len(off) - 1
    return np.sort(np.random.default_rng(seed).choice(P, size=k, replace=False))


def _subset(nodes, off, idx):
    progs = synth.unpack(nodes, off)
    return pack([progs[i] for i in idx])


@pytest.mark.parametrize("name,n_rows", [("pagie_large", 1 << 24), ("pagie_large", 1 << 20),
                                         ("tabular", 10_000_000), ("binary", 1 << 22),
                                         ("wide", 500_000)])
def test_full_size_fitness_sampled(name, n_rows):
    """64 sampled programs of each full-size workload, in the bench's launch
    configuration (the tunables gp_autotune picks for it), against the FP64
    oracle over every row (parity.py: check_fitness_sampled)."""
    k = 64
    wl = synth.workload(name, n_rows=n_rows)
    d = wl.data
    pn, po, dX, dy, dw = put(wl.nodes, wl.offsets, d.X, d.y, d.w)
    opts = gp.gp_autotune(pn, po, dX, dy, dw, metric=wl.metric)
    fit = gp.gp_evaluate_ex(pn, po, dX, dy, dw, metric=wl.metric, opts=opts).cpu().numpy()
    assert np.isfinite(fit).mean() > 0.5
    idx = _sample(wl.offsets, k, 5)
    sn, so = _subset(wl.nodes, wl.offsets, idx)
    strict, cond, flagged = check_fitness_sampled(fit[idx], sn, so, d.X, d.y, d.w, wl.metric)
    assert strict + cond >= k // 2, (name, strict, cond, flagged)
    assert strict >= k // 4, (name, strict, cond, flagged)


def test_accumulators_against_the_oracle_at_10m_rows():
    """The tabular workload (10M rows x 28 columns, RMSE): the fitness with
    FP64 and with Kahan-compensated FP32 cross-chunk sums, each against the
    FP64 oracle over every row on sampled programs: within 1e-4 wherever
    the FP32 error bound certifies the program (check_fitness), and at
    least 8 of them certified."""
    wl = synth.workload("tabular")
    d = wl.data
    pn, po, dX, dy, dw = put(wl.nodes, wl.offsets, d.X, d.y, d.w)
    idx = _sample(wl.offsets, 24, 13)
    sn, so = _subset(wl.nodes, wl.offsets, idx)
    for acc in ("fp64", "kahan32"):
        fit = gp.gp_evaluate_ex(pn, po, dX, dy, dw, metric=wl.metric,
                                opts=gp.make_opts(accum=acc)).cpu().numpy()
        st, _ = check_fitness(fit[idx], sn, so, d.X, d.y, d.w, wl.metric)
        assert st.strict >= 8, (acc, st)


def test_full_size_const_grad_sampled():
    wl = synth.workload("const_tune")
    d = wl.data
    pn, po, dX, dy, _ = put(wl.nodes, wl.offsets, d.X, d.y)
    g, f = gp.gp_const_grad(pn, po, dX, dy, metric="mse")
    g = g.cpu().numpy().astype(np.float64)
    # 48 sampled programs; those whose every row the FP32 bound certifies
    # are compared (strictly, or against their FP32 deviation), at least 8
    # of them strictly
    idx = _sample(wl.offsets, 48, 9)
    sn, so = _subset(wl.nodes, wl.offsets, idx)
    g64, f64, gabs = oracle.const_grad(sn, so, d.X, d.y, None, "mse", with_abs=True)
    g32, _ = oracle.const_grad32(sn, so, d.X, d.y, None, "mse")
    v, e, fl = oracle.predict_bound(sn, so, d.X, ulps_fn=4.0)
    strict, cond = _grad_check(g[idx], g64, g32, gabs, fl, None, e, v)
    assert strict >= 8, (strict, cond, len(idx))
    # the fitness returned beside the gradient is the evaluator's
    fe = gp.gp_evaluate(pn, po, dX, dy, metric="mse").cpu().numpy()
    fc = f.cpu().numpy()
    fin = np.isfinite(fe)
    np.testing.assert_array_equal(np.isfinite(fc), fin)
    np.testing.assert_allclose(fc[fin], fe[fin], rtol=1e-5)
