"""GPU parity of the device mutation step (gp_mutate) with the oracle.

The next population is integer work on Philox streams, so the bar is bit
equality: nodes, offsets and kinds must equal the oracle's for the same
parents, parameters, seed and offset.  Covers the default mix on the
pagie_large population, each kind alone, hoisting under both the 20-slot and
the 255-node bound, restricted function sets, invalid parents, a parent
index out of range, caller workspaces, and whole generations (evaluate,
select, mutate) run back to back on the device.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_2110_11226_gb300 import gp, synth
from parity import check_fitness

pytestmark = pytest.mark.gpu

OP = synth.OP


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(nodes, off, n_feat, parents, seed, offset, **kw):
    pn = gp.nodes_to_device(nodes)
    po = _dev(off.astype(np.int32))
    params = gp.make_mut_params(**kw)
    out, oo, kind = gp.gp_mutate(pn, po, n_feat, _dev(parents.astype(np.int32)), params,
                                 seed=seed, offset=offset)
    oo = oo.cpu().numpy()
    got = gp.nodes_from_device(out[:int(oo[-1])])
    return got, oo, kind.cpu().numpy()


def _check(nodes, off, n_feat, parents, seed=3, offset=0, **kw):
    got, go, gk = _run(nodes, off, n_feat, parents, seed, offset, **kw)
    wn, wo, wk = oracle.mutate(nodes, off, n_feat, parents, seed=seed, offset=offset, **kw)
    np.testing.assert_array_equal(go, wo)
    np.testing.assert_array_equal(gk, wk)
    assert got.tobytes() == wn.tobytes()
    return gk


def test_default_mix_on_the_large_population_is_bit_exact():
    wl = synth.workload("pagie_large", n_rows=1024)
    P = len(wl.offsets) - 1
    parents = np.random.default_rng(1).integers(0, P, 2 * P)
    kind = _check(wl.nodes, wl.offsets, 2, parents, seed=2 ** 33 + 7, offset=5)
    counts = np.bincount(kind, minlength=5)
    assert counts.min() > 50  # every kind occurs


@pytest.mark.parametrize("kind", ["crossover", "subtree", "hoist", "point"])
def test_each_kind_alone(kind):
    nodes, off = synth.ramped_half_and_half(700, 2, 9, synth.EXTENDED_SET, 5, seed=8)
    parents = np.random.default_rng(9).integers(0, 700, 2 * 2000)
    probs = dict(p_crossover=0.0, p_subtree=0.0, p_hoist=0.0, p_point=0.0)
    probs["p_" + kind] = 1.0
    got = _check(nodes, off, 5, parents, seed=11, offset=2 ** 40 + 1, p_replace=0.4,
                 subtree_depth=6, **probs)
    assert np.mean(got == oracle.MUT_KINDS[kind]) > 0.99


def test_hoisting_under_both_bounds_and_restricted_functions():
    deep = [(OP["add"], 0, 0.0)] * 19 + [(OP["var"], 0, 0.0)] * 20     # 20 stack slots
    long = []
    for _ in range(120):
        long += [(OP["mul"], 0, 0.0), (OP["const"], 0, 0.25)]
    long += [(OP["var"], 1, 0.0)]                                        # 241 nodes
    nodes, off = synth.pack([deep, long])
    parents = np.array([0, 1, 1, 0, 1, 1, 0, 0] * 256)
    _check(nodes, off, 2, parents, seed=4, p_crossover=0.6, p_subtree=0.4, p_hoist=0.0,
           p_point=0.0, subtree_depth=6, functions=("add", "sin"))


def test_invalid_parents_and_bad_index():
    good = [(OP["add"], 0, 0.0), (OP["var"], 0, 0.0), (OP["const"], 0, 1.0)]
    leftover = [(OP["var"], 0, 0.0), (OP["var"], 0, 0.0)]
    nodes, off = synth.pack([good, leftover])
    parents = np.array([1, 0, 0, 1] * 40)
    _check(nodes, off, 1, parents, seed=1, p_crossover=1.0, p_subtree=0.0, p_hoist=0.0, p_point=0.0)
    gp.gp_last_device_status()  # clear
    bad = np.array([0, 0, 5, 0, 0, -1], np.int32)
    got, go, gk = _run(nodes, off, 1, bad, 1, 0)
    assert gp.gp_last_device_status() & gp.DEV_BAD_PARENT
    progs = [got[go[t]:go[t + 1]] for t in range(3)]
    for t in (1, 2):
        assert len(progs[t]) == 1 and progs[t][0]["op"] == OP["const"] and progs[t][0]["c"] == 0.0


def test_arguments_and_caller_workspace():
    nodes, off = synth.ramped_half_and_half(50, 2, 5, synth.FULL_SET, 2, seed=1)
    pn, po = gp.nodes_to_device(nodes), _dev(off.astype(np.int32))
    par = _dev(np.random.default_rng(0).integers(0, 50, 100).astype(np.int32))
    need = gp.gp_mutate_workspace_size(50)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    a = gp.gp_mutate(pn, po, 2, par, seed=3, ws=ws)
    b = gp.gp_mutate(pn, po, 2, par, seed=3)
    torch.cuda.synchronize()
    assert torch.equal(a[1], b[1]) and torch.equal(a[0][:int(a[1][-1])], b[0][:int(b[1][-1])])
    with pytest.raises(gp.GPError):
        gp.gp_mutate(pn, po, 2, par, seed=3, ws=ws[:need - 256])
    for bad in (dict(p_crossover=0.9, p_subtree=0.2), dict(subtree_depth=7), dict(functions=()),
                dict(p_replace=1.5)):
        with pytest.raises(gp.GPError):
            gp.gp_mutate(pn, po, 2, par, gp.make_mut_params(**bad))


def test_generations_on_the_device_match_the_oracle():
    """evaluate -> tournament (2 per offspring) -> mutate, three times, all on
    the device; each population equals the oracle's, each fitness vector
    matches the oracle's fitness of that population."""
    d = synth.pagie_data(2048 + 17, 3)
    nodes, off = synth.ramped_half_and_half(256, 2, 6, synth.FULL_SET, 2, seed=21)
    dX, dy = _dev(d.X), _dev(d.y)
    pn, po = gp.nodes_to_device(nodes), _dev(off.astype(np.int32))
    o_nodes, o_off = nodes, off
    for gen in range(3):
        fit = gp.gp_evaluate(pn, po, dX, dy, metric="rmse")
        check_fitness(fit.cpu().numpy(), o_nodes, o_off, d.X, d.y, None, "rmse")
        win = gp.gp_tournament_ex(fit, 2 * 256, 7, seed=100 + gen)
        want_win = oracle.tournament(fit.cpu().numpy(), 2 * 256, 7, 100 + gen)
        np.testing.assert_array_equal(win.cpu().numpy(), want_win)
        out, oo, _ = gp.gp_mutate(pn, po, 2, win, seed=200 + gen, offset=gen)
        o_nodes, o_off, _ = oracle.mutate(o_nodes, o_off, 2, want_win, seed=200 + gen, offset=gen)
        np.testing.assert_array_equal(oo.cpu().numpy(), o_off)
        n = int(o_off[-1])
        pn = out[:n].clone()
        po = oo.clone()
        assert gp.nodes_from_device(pn).tobytes() == o_nodes.tobytes()
