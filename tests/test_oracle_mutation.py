"""Pins of the oracle's mutation step (CPU only).

Each offspring must be what its kind defines (Sec. II-A: crossover, subtree,
hoist and point mutation, reproduction; Sec. III-C2: the hoisted crossover
keeps the child within 20 stack slots), checked here by brute force over the
parent's and donor's subtrees, by invariants (validity, arity patterns,
depth limits) and by the statistics of the draws (kind frequencies, uniform
node choice, the constant distribution), with the first draw of every
offspring recomputed from the Philox generator that the cuRAND pin fixes.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2110_11226_gb300 import synth

OP = synth.OP
ARITY = synth.ARITY
KIND = oracle.MUT_KINDS


def _progs(nodes, off):
    return [nodes[off[p]:off[p + 1]] for p in range(len(off) - 1)]


def _sizes(prog):
    """Subtree size of every node of a prefix list."""
    n = len(prog)
    size = np.zeros(n, np.int64)
    stack = []
    for i in range(n - 1, -1, -1):
        a = ARITY[int(prog[i]["op"])]
        s = 1
        for _ in range(a):
            s += stack.pop()
        size[i] = s
        stack.append(s)
    return size


def _depth(prog):
    return synth.tree_depth([(int(n["op"]), int(n["feat"]), float(n["c"])) for n in prog])


def _key(prog):
    return prog.tobytes()


def _splices(par, don, proper=False):
    """Every child obtained by replacing one subtree of par with one subtree
    of don (with proper=True and don == par: a proper sub-subtree of the
    replaced one, as hoist mutation does)."""
    sp, sd = _sizes(par), _sizes(don)
    out = set()
    for i in range(len(par)):
        if proper:
            ks = range(i + 1, i + sp[i]) if sp[i] > 1 else [i]
        else:
            ks = range(len(don))
        for k in ks:
            child = np.concatenate([par[:i], don[k:k + sd[k]], par[i + sp[i]:]])
            out.add(_key(child))
    return out


def _population(n, seed, depth=(2, 7), n_feat=3):
    return synth.ramped_half_and_half(n, depth[0], depth[1], synth.FULL_SET, n_feat, seed=seed)


def _valid(prog, n_feat):
    st, hw = oracle.validate(prog, n_feat)
    return st == oracle.OK and hw <= 20 and len(prog) <= 255


def test_children_are_valid_and_kinds_follow_the_first_draw():
    nodes, off = _population(400, 1)
    rng = np.random.default_rng(2)
    parents = rng.integers(0, 400, 2 * 3000).astype(np.int32)
    probs = dict(p_crossover=0.5, p_subtree=0.15, p_hoist=0.1, p_point=0.15)
    seed, offset = 2 ** 40 + 3, 17
    cn, co, kind = oracle.mutate(nodes, off, 3, parents, seed=seed, offset=offset, **probs)
    assert len(co) == 3001 and co[0] == 0 and np.all(np.diff(co) >= 1)
    for c in _progs(cn, co):
        assert _valid(c, 3)
    # the kind is decided by word 0 of the offspring's Philox stream
    cum = np.cumsum([probs["p_crossover"], probs["p_subtree"], probs["p_hoist"], probs["p_point"]])
    thr = np.minimum(np.floor(cum * 2.0 ** 32), 2.0 ** 32)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for t in range(3000):
        u0 = int(oracle.philox4x32_10([0, t, offset & 0xFFFFFFFF, offset >> 32], key)[0])
        want = next((q + 1 for q in range(4) if u0 < thr[q]), 0)
        assert kind[t] == want, t
    # and the kinds' frequencies follow the probabilities (5 sigma)
    n = len(kind)
    for name, p in (("crossover", 0.5), ("subtree", 0.15), ("hoist", 0.1), ("point", 0.15),
                    ("reproduction", 0.1)):
        k = int(np.sum(kind == KIND[name]))
        assert abs(k - n * p) < 5 * math.sqrt(n * p * (1 - p)), name


def test_each_kind_is_what_it_defines():
    nodes, off = _population(60, 3, depth=(1, 5))
    progs = _progs(nodes, off)
    rng = np.random.default_rng(4)
    parents = rng.integers(0, 60, 2 * 600).astype(np.int32)
    funcs = ("add", "mul", "sin", "neg")
    cn, co, kind = oracle.mutate(nodes, off, 3, parents, p_crossover=0.3, p_subtree=0.2,
                                 p_hoist=0.2, p_point=0.2, p_replace=0.3, subtree_depth=3,
                                 functions=funcs, seed=9)
    children = _progs(cn, co)
    allowed = {OP[f] for f in funcs}
    seen = set()
    for t, c in enumerate(children):
        par, don = progs[parents[2 * t]], progs[parents[2 * t + 1]]
        k = int(kind[t])
        seen.add(k)
        if k == KIND["reproduction"]:
            assert _key(c) == _key(par)
        elif k == KIND["hoist"]:
            assert _key(c) in _splices(par, par, proper=True)
        elif k == KIND["crossover"]:
            # some subtree of the parent replaced by some subtree of the
            # donor (the drawn one or one hoisted out of it)
            assert _key(c) in _splices(par, don)
        elif k == KIND["point"]:
            assert len(c) == len(par)
            for a, b in zip(par, c):
                ar = ARITY[int(a["op"])]
                assert ARITY[int(b["op"])] == ar
                if ar > 0 and b["op"] != a["op"]:
                    assert int(b["op"]) in allowed
        elif k == KIND["subtree"]:
            # the parent with one subtree replaced by a grow tree of depth
            # <= 3 over the allowed functions (or a part of one)
            sp = _sizes(par)
            ok = False
            for i in range(len(par)):
                pre, post = par[:i], par[i + sp[i]:]
                if len(c) < len(pre) + len(post) + 1:
                    continue
                if _key(c[:i]) != _key(pre) or (len(post) and _key(c[len(c) - len(post):]) != _key(post)):
                    continue
                mid = c[i:len(c) - len(post)]
                if len(_sizes(mid)) and _sizes(mid)[0] == len(mid) and _depth(mid) <= 3 and \
                        all(ARITY[int(n["op"])] == 0 or int(n["op"]) in allowed for n in mid):
                    ok = True
                    break
            assert ok, t
        assert _valid(c, 3)
    assert seen == set(KIND.values())


def test_hoisted_crossover_keeps_children_within_the_stack():
    # parents that already need 20 slots and 200+ nodes, donors with deep,
    # long subtrees: a plain splice would overflow either bound
    deep = [(OP["add"], 0, 0.0)] * 19 + [(OP["var"], 0, 0.0)] * 20  # right spine: 20 slots
    long = []
    for _ in range(100):
        long += [(OP["add"], 0, 0.0), (OP["const"], 0, 0.5)]
    long += [(OP["var"], 0, 0.0)]
    nodes, off = synth.pack([deep, long])
    assert oracle.validate(nodes[off[0]:off[1]], 1)[1] == 20
    parents = np.array([0, 1, 1, 0] * 300, np.int32)
    cn, co, kind = oracle.mutate(nodes, off, 1, parents, p_crossover=1.0, p_subtree=0.0,
                                 p_hoist=0.0, p_point=0.0, seed=5)
    assert np.all(kind == KIND["crossover"])
    progs = _progs(nodes, off)
    reachable = {(a, b): _splices(progs[a], progs[b]) for a, b in ((0, 1), (1, 0))}
    for t, c in enumerate(_progs(cn, co)):
        assert _valid(c, 1)
        assert _key(c) in reachable[(int(parents[2 * t]), int(parents[2 * t + 1]))]


def test_hoist_node_choice_is_uniform():
    # a full binary tree whose leaves are distinct constants: the child
    # identifies the replaced node i and the hoisted node k
    def full(d, leaves):
        if d == 0:
            return [(OP["const"], 0, float(leaves.pop()))]
        return [(OP["add"], 0, 0.0)] + full(d - 1, leaves) + full(d - 1, leaves)
    prog = full(3, list(range(1, 9)))  # 15 nodes
    nodes, off = synth.pack([prog])
    par = nodes
    cands = {}
    sp = _sizes(par)
    internal = [i for i in range(15) if sp[i] > 1]
    for i in internal:
        for k in range(i + 1, i + sp[i]):
            child = np.concatenate([par[:i], par[k:k + sp[k]], par[i + sp[i]:]])
            assert _key(child) not in cands
            cands[_key(child)] = (i, k)
    n = 6000
    cn, co, kind = oracle.mutate(nodes, off, 1, np.zeros(2 * n, np.int32), p_crossover=0.0,
                                 p_subtree=0.0, p_hoist=1.0, p_point=0.0, seed=11)
    # a leaf (8 of 15 nodes) hoists nothing: the child is the parent
    picks = [cands.get(_key(c), (-1, -1)) for c in _progs(cn, co)]
    counts = np.bincount([i + 1 for i, _ in picks], minlength=16)
    want = np.array([8 / 15] + [1 / 15 if i in internal else 0 for i in range(15)]) * n
    live = want > 0
    chi2 = np.sum((counts[live] - want[live]) ** 2 / want[live])
    assert counts[~live].sum() == 0
    assert chi2 < 40  # 7 degrees of freedom, p ~ 1e-6
    # k is uniform over the proper descendants of the root (node 0)
    k_root = np.bincount([k for i, k in picks if i == 0], minlength=15)[1:]
    e = k_root.sum() / 14
    assert np.sum((k_root - e) ** 2 / e) < 45  # 13 degrees of freedom


def test_point_mutation_rate_and_new_terminals():
    nodes, off = _population(200, 6, n_feat=4)
    rng = np.random.default_rng(7)
    parents = rng.integers(0, 200, 2 * 2000).astype(np.int32)
    cn, co, kind = oracle.mutate(nodes, off, 4, parents, p_crossover=0.0, p_subtree=0.0,
                                 p_hoist=0.0, p_point=1.0, p_replace=0.25,
                                 functions=("add", "sub", "mul", "div", "sin", "cos"), seed=3)
    progs = _progs(nodes, off)
    changed = total = 0
    consts = []
    term_kinds = np.zeros(5, np.int64)  # var 0..3, const
    for t, c in enumerate(_progs(cn, co)):
        par = progs[parents[2 * t]]
        total += len(par)
        for a, b in zip(par, c):
            changed += a.tobytes() != b.tobytes()
            if ARITY[int(a["op"])] == 0 and a.tobytes() != b.tobytes():
                if b["op"] == OP["const"]:
                    consts.append(float(b["c"]))
                    term_kinds[4] += 1
                else:
                    term_kinds[int(b["feat"])] += 1
    # a replaced node can draw its own value again (functions: 1 in 4 for
    # binary, 1 in 2 for unary; terminals almost never), so the observed
    # rate is a little under 0.25
    assert 0.17 < changed / total < 0.25
    consts = np.array(consts)
    assert consts.min() >= -1.0 and consts.max() < 1.0
    assert np.all(consts * 2 ** 23 == np.round(consts * 2 ** 23))
    assert abs(consts.mean()) < 5 / math.sqrt(12 * len(consts)) * 2
    # a new terminal is variable f (each 1/5) or a constant (1/5)
    e = term_kinds.sum() / 5
    assert np.sum((term_kinds - e) ** 2 / e) < 25


def test_invalid_parents_and_arguments():
    good = [(OP["add"], 0, 0.0), (OP["var"], 0, 0.0), (OP["const"], 0, 1.0)]
    leftover = [(OP["var"], 0, 0.0), (OP["var"], 0, 0.0)]
    nodes, off = synth.pack([good, leftover])
    par = np.array([1, 0, 0, 1] * 50, np.int32)
    cn, co, kind = oracle.mutate(nodes, off, 1, par, p_crossover=1.0, p_subtree=0.0,
                                 p_hoist=0.0, p_point=0.0, seed=1)
    kids = _progs(cn, co)
    progs = _progs(nodes, off)
    for t in range(100):
        # an invalid parent is copied; an invalid donor leaves the parent
        assert kind[t] == KIND["reproduction"]
        assert _key(kids[t]) == _key(progs[par[2 * t]])
    with pytest.raises(ValueError):
        oracle.mutate(nodes, off, 1, np.array([0, 2], np.int32))
    with pytest.raises(ValueError):
        oracle.mutate(nodes, off, 1, np.array([0, 0], np.int32), p_crossover=0.8, p_subtree=0.5)
    with pytest.raises(ValueError):
        oracle.mutate(nodes, off, 1, np.array([0, 0], np.int32), functions=())


def test_streams_are_reproducible_and_distinct():
    nodes, off = _population(100, 8)
    parents = np.random.default_rng(0).integers(0, 100, 400).astype(np.int32)
    a = oracle.mutate(nodes, off, 3, parents, seed=5, offset=1)
    b = oracle.mutate(nodes, off, 3, parents, seed=5, offset=1)
    c = oracle.mutate(nodes, off, 3, parents, seed=5, offset=2)
    assert a[0].tobytes() == b[0].tobytes() and np.array_equal(a[1], b[1])
    assert a[0].tobytes() != c[0].tobytes()
