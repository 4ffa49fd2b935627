"""Argument checks of the Python binding (CPU): the library reads and writes
through raw pointers, so the binding refuses a wrong element type or a
too-short tensor before any call reaches the library, and it refuses host
tensors outright (there is no CPU path behind it)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2110_11226_gb300 import gp, synth


def _problem(n_rows=300, n_progs=8):
    d = synth.pagie_data(n_rows, 1)
    nodes, off = synth.ramped_half_and_half(n_progs, 2, 4, synth.BASIC_SET, 2, seed=3)
    pn = torch.from_numpy(np.ascontiguousarray(nodes).view(np.int64).copy())
    return (pn, torch.from_numpy(off.astype(np.int32)), torch.from_numpy(d.X),
            torch.from_numpy(d.y), torch.ones(n_rows, dtype=torch.float32))


class _Recorder:
    """Stands in for libgp: records which entry points were called and
    returns GP_OK without touching any pointer."""

    def __init__(self):
        self.called = []

    def __getattr__(self, name):
        def call(*args):
            self.called.append(name)
            return 0
        return call


@pytest.fixture
def lib(monkeypatch):
    """Host tensors stand in for device ones and the library is a recorder,
    so only the binding's own checks run."""
    stub = _Recorder()
    monkeypatch.setattr(gp, "_on_device", lambda t: True)
    monkeypatch.setattr(gp, "_lib", stub)
    monkeypatch.setattr(gp, "_stream", lambda s: None)
    return stub


def test_host_tensors_are_refused():
    pn, po, X, y, w = _problem()
    with pytest.raises(TypeError, match="must be a CUDA tensor"):
        gp.gp_evaluate(pn, po, X, y, w, out=torch.empty(po.numel() - 1))
    with pytest.raises(TypeError, match="must be a CUDA tensor"):
        gp.gp_tournament_ex(torch.empty(4), 4, 2, 0)


def test_well_formed_arguments_reach_the_library(lib):
    pn, po, X, y, w = _problem()
    P = po.numel() - 1
    i32 = dict(dtype=torch.int32)
    calls = {
        "gp_evaluate": lambda: gp.gp_evaluate(pn, po, X, y, w, out=torch.empty(P)),
        "gp_evaluate_static": lambda: gp.gp_evaluate_static(pn, po, X, y, w, out=torch.empty(P)),
        "gp_evaluate_plain": lambda: gp.gp_evaluate_plain(pn, po, X, y, w, out=torch.empty(P)),
        "gp_evaluate_ex": lambda: gp.gp_evaluate_ex(
            pn, po, X, y, w, out=torch.empty(P), out64=torch.empty(P, dtype=torch.float64),
            out_status=torch.empty(P, **i32), ws=torch.empty(1024, dtype=torch.uint8)),
        "gp_predict": lambda: gp.gp_predict(pn, po, X, out=torch.empty(P, X.shape[1])),
        "gp_predict_ex": lambda: gp.gp_predict_ex(pn, po, X, gp.make_opts(rows_per_thread=8),
                                                  out=torch.empty(P, X.shape[1])),
        "gp_const_grad": lambda: gp.gp_const_grad(pn, po, X, y, w,
                                                  out_grad=torch.empty(P, gp.MAX_CONSTS),
                                                  out_fitness=torch.empty(P)),
        "gp_adam_step": lambda: gp.gp_adam_step(pn, po, torch.empty(P, 16), torch.zeros(P, 16),
                                                torch.zeros(P, 16), 1),
        "gp_get_consts": lambda: gp.gp_get_consts(pn, po, out=torch.empty(P, 16)),
        "gp_set_consts": lambda: gp.gp_set_consts(pn, po, torch.zeros(P, 16)),
        "gp_tournament_ex": lambda: gp.gp_tournament_ex(torch.empty(P), 5, 3, 1, offsets=po,
                                                        out=torch.empty(5, **i32)),
        "gp_tournament": lambda: gp.gp_tournament(torch.empty(P), 3, 1, out=torch.empty(P, **i32)),
        "gp_mutate": lambda: gp.gp_mutate(pn, po, 2, torch.zeros(2 * P, **i32),
                                          out=torch.empty(P * 255, dtype=torch.int64),
                                          out_offsets=torch.empty(P + 1, **i32),
                                          out_kind=torch.empty(P, **i32),
                                          ws=torch.empty(1024, dtype=torch.uint8)),
        "gp_autotune": lambda: gp.gp_autotune(pn, po, X, y, w),
    }
    for name, call in calls.items():
        call()
        assert lib.called[-1] == name
    # y and w may be longer than X's rows (the library reads the first n_rows)
    gp.gp_evaluate(pn, po, X, torch.cat([y, y]), torch.cat([w, w]), out=torch.empty(P))
    # outputs the binding allocates itself meet its own checks
    gp.gp_mutate(pn, po, 2, torch.zeros(2 * P, **i32))
    gp.gp_const_grad(pn, po, X, y)
    assert lib.called[-3:] == ["gp_evaluate", "gp_mutate", "gp_const_grad"]


def test_wrong_element_types_are_refused(lib):
    pn, po, X, y, w = _problem()
    P = po.numel() - 1
    cases = [
        (lambda: gp.gp_evaluate(pn, po, X.double(), y), "X must be torch.float32"),
        (lambda: gp.gp_evaluate(pn, po, X, y.double()), "y must be torch.float32"),
        (lambda: gp.gp_evaluate(pn, po, X, y, w.half()), "w must be torch.float32"),
        (lambda: gp.gp_evaluate(pn, po.long(), X, y), "offsets must be torch.int32"),
        (lambda: gp.gp_evaluate(pn.view(torch.float64), po, X, y), "progs must be torch.int64"),
        (lambda: gp.gp_evaluate(pn, po, X, y, out=torch.empty(P, dtype=torch.float64)),
         "out must be torch.float32"),
        (lambda: gp.gp_evaluate_ex(pn, po, X, y, out=torch.empty(P), out64=torch.empty(P)),
         "out64 must be torch.float64"),
        (lambda: gp.gp_tournament_ex(torch.empty(P, dtype=torch.float64), 4, 2, 0), "fitness"),
        (lambda: gp.gp_mutate(pn, po, 2, torch.zeros(2 * P, dtype=torch.int64)), "parents"),
    ]
    for call, msg in cases:
        with pytest.raises(TypeError, match=msg):
            call()
    assert lib.called == []


def test_short_tensors_are_refused(lib):
    pn, po, X, y, w = _problem(n_rows=300)
    P = po.numel() - 1
    i32 = dict(dtype=torch.int32)
    cases = [
        (lambda: gp.gp_evaluate(pn, po, X, y[:299]), "y holds 299"),
        (lambda: gp.gp_evaluate(pn, po, X, y, w[:10]), "w holds 10"),
        (lambda: gp.gp_evaluate(pn, po, X, y, out=torch.empty(P - 1)), "out holds"),
        (lambda: gp.gp_evaluate_ex(pn, po, X, y, out=torch.empty(P),
                                   out_status=torch.empty(1, **i32)), "out_status"),
        (lambda: gp.gp_predict(pn, po, X, out=torch.empty(P, 299)), "out holds"),
        (lambda: gp.gp_const_grad(pn, po, X, y, out_grad=torch.empty(P, 15)), "out_grad"),
        (lambda: gp.gp_adam_step(pn, po, torch.empty(P, 16), torch.zeros(P, 8),
                                 torch.zeros(P, 16), 1), "m holds"),
        (lambda: gp.gp_tournament_ex(torch.empty(P), 9, 2, 0, out=torch.empty(8, **i32)),
         "out holds 8"),
        (lambda: gp.gp_tournament_ex(torch.empty(P), 4, 2, 0, offsets=po[:-1]), "offsets holds"),
        (lambda: gp.gp_mutate(pn, po, 2, torch.zeros(2 * P, **i32),
                              out=torch.empty(P * 254, dtype=torch.int64)), "out holds"),
    ]
    for call, msg in cases:
        with pytest.raises(ValueError, match=msg):
            call()
    assert lib.called == []
