"""gp_evaluate_static: fitness without any device allocation.

Some callers cannot allocate device memory when they evaluate (their memory
is handed out at start-up to another allocator, or they must not call
cudaMalloc/cudaFree because those can synchronise the device).  This entry
point uses the library's fixed scratch array instead; here it must give the
same fitness as gp_evaluate on two calls in a row, with different inputs so
that nothing of the first call can carry into the second, and must refuse a
problem too large for the array without launching anything.

The file is named to be collected last: its first call on the device does
the one-time address look-up of the scratch array.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

from paper_2110_11226_gb300 import gp, synth

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _call_static(pn, po, dX, dy, dw, metric, out):
    """Through the C ABI directly: gp_evaluate_static(...) -> status."""
    lib = ctypes.CDLL(gp.LIB_PATH)
    f = lib.gp_evaluate_static
    P = ctypes.c_void_p
    f.restype = ctypes.c_int
    f.argtypes = [P, P, ctypes.c_int, P, ctypes.c_int64, ctypes.c_int, P, P, ctypes.c_int, P, P]
    ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return f(ptr(pn), ptr(po), int(po.numel()) - 1, ptr(dX), int(dX.shape[1]), int(dX.shape[0]),
             ptr(dy), ptr(dw), gp.METRICS[metric], ptr(out), stream)


def test_static_entry_matches_gp_evaluate_twice():
    cases = [
        (synth.workload("pagie_large", n_rows=(1 << 17) + 37, n_progs=1024), "rmse"),
        (synth.workload("binary", n_rows=50_000, n_progs=300), "logloss"),
    ]
    for wl, metric in cases:
        d = wl.data
        pn = gp.nodes_to_device(wl.nodes)
        po = _dev(wl.offsets)
        dX, dy = _dev(d.X), _dev(d.y)
        dw = None if d.w is None else _dev(d.w)
        out = torch.full((len(wl.offsets) - 1,), -1.0, device="cuda")
        assert _call_static(pn, po, dX, dy, dw, metric, out) == 0
        ref = gp.gp_evaluate(pn, po, dX, dy, dw, metric=metric)
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        np.testing.assert_array_equal(np.isfinite(a), np.isfinite(b))
        fin = np.isfinite(b)
        np.testing.assert_allclose(a[fin], b[fin], rtol=1e-6)


def test_static_entry_refuses_a_problem_beyond_its_scratch():
    # 16384 programs need 32 MiB of compiled code alone
    nodes, off = synth.ramped_half_and_half(16384, 1, 2, synth.BASIC_SET, 2, seed=1)
    d = synth.pagie_data(1024, 2)
    out = torch.zeros(16384, device="cuda")
    rc = _call_static(gp.nodes_to_device(nodes), _dev(off), _dev(d.X), _dev(d.y), None, "mse", out)
    assert rc == -7  # GP_ERR_WORKSPACE
    torch.cuda.synchronize()
    assert torch.all(out == 0)
