"""The seeded input generators (CPU): the tree helpers agree with recursive
definitions and with the oracle's validator, ramped half-and-half keeps its
depth ramp, methods and caps, the terminal mix follows its probabilities,
and each dataset is what its recipe says (Pagie-1 target, heavy-tailed
columns, noise level, class weights, label flips), reproducibly."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2110_11226_gb300 import synth

OP, ARITY = synth.OP, synth.ARITY


def _tree(prog, pos=0):
    """(end position, depth, leaf depths) of the subtree starting at pos."""
    a = ARITY[prog[pos][0]]
    if a == 0:
        return pos + 1, 0, [0]
    end, depth, leaves = pos + 1, 0, []
    for _ in range(a):
        end, d, lv = _tree(prog, end)
        depth = max(depth, d + 1)
        leaves += [x + 1 for x in lv]
    return end, depth, leaves


def _value(prog, X, pos=0):
    """FP64 value of a tree over {add, sub, mul, sin, cos, abs, neg}."""
    op, feat, c = prog[pos]
    name = synth.OP_NAME[op]
    if name == "const":
        return pos + 1, np.full(X.shape[1], float(np.float32(c)))
    if name == "var":
        return pos + 1, X[feat].astype(np.float64)
    end, a = _value(prog, X, pos + 1)
    if ARITY[op] == 1:
        return end, {"sin": np.sin, "cos": np.cos, "abs": np.abs, "neg": np.negative}[name](a)
    end, b = _value(prog, X, end)
    return end, {"add": a + b, "sub": a - b, "mul": a * b}[name]


def test_tree_helpers_agree_with_recursion_and_the_oracle():
    nodes, off = synth.random_programs(400, 9, synth.EXTENDED_SET, 3, seed=17)
    for prog in synth.unpack(nodes, off):
        end, depth, _ = _tree(prog)
        assert end == len(prog)
        assert synth.tree_depth(prog) == depth
        packed, _ = synth.pack([prog])
        st, hw = oracle.validate(packed, 3)
        assert st == oracle.OK and synth.stack_high_water(prog) == hw
    # pack / unpack round trip, offsets an exclusive scan of the lengths
    progs = synth.unpack(nodes, off)
    n2, o2 = synth.pack(progs)
    assert n2.tobytes() == nodes.tobytes() and np.array_equal(o2, off)
    assert off[0] == 0 and np.array_equal(np.diff(off), [len(p) for p in progs])


def test_ramped_half_and_half_ramp_and_methods():
    dmin, dmax, P = 2, 6, 200
    nodes, off = synth.ramped_half_and_half(P, dmin, dmax, synth.FULL_SET, 2, seed=5)
    n_d = dmax - dmin + 1
    seen = set()
    for i, prog in enumerate(synth.unpack(nodes, off)):
        d = dmin + i % n_d
        _, depth, leaves = _tree(prog)
        if (i // n_d) % 2 == 0:          # full: every leaf at the target depth
            assert depth == d and set(leaves) == {d}
            seen.add(("full", d))
        else:                            # grow: no deeper than the target
            assert depth <= d
            seen.add(("grow", d))
        assert len(prog) <= synth.MAX_LEN and synth.stack_high_water(prog) <= synth.MAX_STACK
    assert len(seen) == 2 * n_d


def test_length_and_constant_caps():
    nodes, off = synth.ramped_half_and_half(300, 4, 10, synth.FULL_SET, 2, seed=103,
                                            max_consts=16)
    progs = synth.unpack(nodes, off)
    assert max(len(p) for p in progs) <= 255
    assert max(sum(n[0] == OP["const"] for n in p) for p in progs) <= 16
    # depth-10 full trees exist within the cap (unary functions keep them short)
    assert any(_tree(p)[1] == 10 for p in progs)
    with pytest.raises(RuntimeError):
        synth.ramped_half_and_half(1, 9, 9, synth.BASIC_SET, 2, seed=1)  # 1023 nodes, never fits


def test_terminal_mix_follows_its_probabilities():
    n_feat = 3
    nodes, off = synth.ramped_half_and_half(3000, 1, 5, synth.BASIC_SET, n_feat, seed=11)
    term = nodes[(nodes["op"] == OP["var"]) | (nodes["op"] == OP["const"])]
    is_var = term["op"] == OP["var"]
    n = len(term)
    p = n_feat / (n_feat + 1.0)
    assert abs(is_var.mean() - p) < 4 * np.sqrt(p * (1 - p) / n)
    counts = np.bincount(term["feat"][is_var], minlength=n_feat)
    assert len(counts) == n_feat and counts.min() > 0.9 * counts.mean()
    c = term["c"][~is_var]
    assert c.min() >= -1.0 and c.max() < 1.0 and abs(c.mean()) < 0.05
    # grow: a node above the depth limit is a terminal with probability 2 / (2 + F)
    g = synth.ramped_half_and_half(4000, 2, 2, synth.BASIC_SET, n_feat, seed=12)
    roots_grow = [p for i, p in enumerate(synth.unpack(*g)) if (i // 1) % 2 == 1]
    root_term = np.mean([ARITY[p[0][0]] == 0 for p in roots_grow])
    q = 2.0 / (2.0 + len(synth.BASIC_SET))
    assert abs(root_term - q) < 4 * np.sqrt(q * (1 - q) / len(roots_grow))


def test_pagie_data_is_the_pagie_polynomial():
    d = synth.pagie_data(20000, 3)
    assert d.X.dtype == np.float32 and d.X.shape == (2, 20000) and d.w is None
    assert d.X.min() >= -5.0 and d.X.max() <= 5.0
    x = d.X.astype(np.float64)
    nz = np.all(x != 0, axis=0)
    want = 1.0 / (1.0 + x[0, nz] ** -4) + 1.0 / (1.0 + x[1, nz] ** -4)   # Eq. pagie as printed
    np.testing.assert_allclose(d.y[nz], want, rtol=2 ** -23, atol=0)
    np.testing.assert_array_equal(d.y, synth.pagie_data(20000, 3).y)


def test_tabular_data_recipe():
    d = synth.tabular_data(40000, 1236)
    assert d.X.shape == (28, 40000) and d.X.dtype == np.float32
    x = d.X.astype(np.float64)
    kurt = ((x - x.mean(1, keepdims=True)) ** 4).mean(1) / x.var(1) ** 2 - 3.0
    assert np.all(kurt[:4] > 1.0) and np.all(np.abs(kurt[4:]) < 0.2)  # Student-t(3) vs N(0,1)
    hid = synth.unpack(*d.hidden)[0]
    _, depth, _ = _tree(hid)
    assert depth == 6 and all(n[1] < 8 for n in hid if n[0] == OP["var"])
    _, h = _value(hid, x)
    ratio = np.std(d.y - h) / np.std(h)
    assert 0.09 < ratio < 0.11


def test_classification_data_recipe():
    d = synth.classification_data(100000, 1237)
    assert d.X.shape == (50, 100000) and d.X.min() >= -1.0 and d.X.max() <= 1.0
    assert set(np.unique(d.y)) <= {0.0, 1.0}
    np.testing.assert_array_equal(d.w, np.where(d.y == 1.0, 1.0, 3.0).astype(np.float32))
    hid = synth.unpack(*d.hidden)[0]
    _, h = _value(hid, d.X.astype(np.float64))
    flipped = np.mean((h > 0).astype(np.float32) != d.y)
    assert abs(flipped - 0.05) < 4 * np.sqrt(0.05 * 0.95 / len(h))


@pytest.mark.parametrize("name,metric,k,funcs,n_progs,n_feat", [
    ("pagie_small", "mse", 20, synth.BASIC_SET, 512, 2),
    ("pagie_large", "rmse", 20, synth.FULL_SET, 4096, 2),
    ("tabular", "rmse", 20, synth.FULL_SET, 2048, 28),
    ("binary", "logloss", 10, synth.FULL_SET, 1024, 50),
    ("const_tune", "mse", 20, synth.FULL_SET, 2048, 2),
])
def test_named_workloads(name, metric, k, funcs, n_progs, n_feat):
    a = synth.workload(name, n_rows=2048)
    b = synth.workload(name, n_rows=2048)
    assert (a.metric, a.tourn_size, a.funcs) == (metric, k, funcs)
    assert len(a.offsets) - 1 == n_progs and a.data.n_feat == n_feat and a.data.n_rows == 2048
    assert a.nodes.tobytes() == b.nodes.tobytes() and a.data.X.tobytes() == b.data.X.tobytes()
    used = set(synth.OP_NAME[o] for o in np.unique(a.nodes["op"])) - {"const", "var"}
    assert used <= set(funcs)
    if name == "const_tune":
        assert max(oracle.count_consts(p) for p in np.split(a.nodes, a.offsets[1:-1])) <= 16
