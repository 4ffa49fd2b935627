"""gp_evaluate_static: fitness without any device allocation.

Some callers cannot allocate device memory when they evaluate (their memory
is handed out at start-up to another allocator, or they must not call
cudaMalloc/cudaFree because those can synchronise the device).  This entry
point uses the library's fixed scratch array instead; here it must give the
same fitness as gp_evaluate, bit for bit, on two calls in a row, with
different inputs so that nothing of the first call can carry into the
second; where the default workspace is too large it must equal
gp_evaluate_ex at the longer row chunks it falls back to; and it must refuse
a problem too large for the array without launching anything.

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


def _same_bits(a, b):
    nan = np.isnan(b)
    np.testing.assert_array_equal(np.isnan(a), nan)
    np.testing.assert_array_equal(a[~nan].view(np.uint32), b[~nan].view(np.uint32))


def test_static_entry_matches_gp_evaluate_twice():
    """Problems whose default workspace fits the array: the fitness is
    gp_evaluate's, bit for bit, on two calls in a row."""
    cases = [
        (synth.workload("pagie_large", n_rows=(1 << 17) + 37, n_progs=1024), "rmse"),
        (synth.workload("binary", n_rows=50_000, n_progs=300), "logloss"),
    ]
    for wl, metric in cases:
        d = wl.data
        P = len(wl.offsets) - 1
        assert gp.gp_static_opts(P, d.n_rows, d.n_feat, metric).chunk_rows == 0
        pn = gp.nodes_to_device(wl.nodes)
        po = _dev(wl.offsets)
        dX, dy = _dev(d.X), _dev(d.y)
        dw = None if d.w is None else _dev(d.w)
        out = torch.full((P,), -1.0, device="cuda")
        assert _call_static(pn, po, dX, dy, dw, metric, out) == 0
        ref = gp.gp_evaluate(pn, po, dX, dy, dw, metric=metric)
        torch.cuda.synchronize()
        _same_bits(out.cpu().numpy(), ref.cpu().numpy())


@pytest.mark.parametrize("n_rows,metric", [(1 << 24, "rmse"), (1 << 22, "pearson")])
def test_static_entry_falls_back_to_longer_chunks(n_rows, metric):
    """Problems whose default workspace exceeds the 16 MiB array (4096
    programs: 16M rows of RMSE partials, or 4M rows of Pearson's FP64
    moments): the call takes longer row chunks, its fitness equals
    gp_evaluate_ex with those chunks bit for bit, and sampled programs
    agree with the oracle over every row."""
    from parity import check_fitness_sampled, check_pearson
    wl = synth.workload("pagie_large", n_rows=n_rows, n_progs=4096)
    d = wl.data
    P = len(wl.offsets) - 1
    opts = gp.gp_static_opts(P, d.n_rows, d.n_feat, metric)
    assert opts.chunk_rows >= 65536, opts.chunk_rows
    default = gp.gp_resolve_opts(P, d.n_rows, d.n_feat)
    assert default.chunk_rows < opts.chunk_rows
    pn = gp.nodes_to_device(wl.nodes)
    po = _dev(wl.offsets)
    dX, dy = _dev(d.X), _dev(d.y)
    out = torch.full((P,), -1.0, device="cuda")
    assert _call_static(pn, po, dX, dy, None, metric, out) == 0
    ref = gp.gp_evaluate_ex(pn, po, dX, dy, None, metric=metric, opts=opts)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    _same_bits(got, ref.cpu().numpy())
    sample = np.random.default_rng(7).choice(P, size=8, replace=False)
    sub = [synth.unpack(wl.nodes, wl.offsets)[i] for i in sample]
    sn, so = synth.pack(sub)
    if metric == "pearson":
        st, _ = check_pearson(got[sample], sn, so, d.X, d.y, None)
        assert st.strict + st.conditioning >= 4, st
    else:
        strict, cond, flagged = check_fitness_sampled(got[sample], sn, so, d.X, d.y, None, metric)
        assert strict + cond >= 4, (strict, cond, flagged)


def test_static_entry_refuses_a_problem_beyond_its_scratch():
    # 16384 programs need 32 MiB of compiled code alone
    nodes, off = synth.ramped_half_and_half(16384, 1, 2, synth.BASIC_SET, 2, seed=1)
    d = synth.pagie_data(1024, 2)
    out = torch.zeros(16384, device="cuda")
    rc = _call_static(gp.nodes_to_device(nodes), _dev(off), _dev(d.X), _dev(d.y), None, "mse", out)
    assert rc == -7  # GP_ERR_WORKSPACE
    torch.cuda.synchronize()
    assert torch.all(out == 0)
