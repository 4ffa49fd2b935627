"""Python binding of libgp (include/gp.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Device arrays
are CUDA torch tensors (PyTorch provides device memory and streams; all
computation runs in libgp's kernels); host arrays are numpy arrays.  There
is no fallback: if libgp.so cannot be built or loaded, importing this module
raises.

Program populations travel as one flat array of 8-byte nodes (int16 op,
int16 feat, float32 c) plus int32 offsets[P+1] (Sec. III-A prefix lists);
``nodes_to_device`` turns the numpy form into a CUDA int64 tensor holding
the same bytes.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np
import torch

from . import build as _build

METRICS = {"mae": 0, "mse": 1, "rmse": 2, "logloss": 3, "pearson": 4, "spearman": 5}
GREATER_IS_BETTER = {"pearson", "spearman"}
ACCUM = {"fp64": 0, "kahan32": 1}
MAX_CONSTS = 16
NODE_DTYPE = np.dtype([("op", "<i2"), ("feat", "<i2"), ("c", "<f4")])

DEV_BAD_PROGRAM = 0x1
DEV_TOO_MANY_CONSTS = 0x2
DEV_QUEUE_CAP = 0x4
DEV_BAD_PARENT = 0x8


class GPError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} failed: {code} ({_lib.gp_status_string(code).decode()})")
        self.code = code


class MutParams(C.Structure):
    _fields_ = [("p_crossover", C.c_float), ("p_subtree", C.c_float), ("p_hoist", C.c_float),
                ("p_point", C.c_float), ("p_point_replace", C.c_float),
                ("subtree_depth", C.c_int), ("functions", C.c_uint32),
                ("reserved", C.c_int * 4)]


MUT_KINDS = {"reproduction": 0, "crossover": 1, "subtree": 2, "hoist": 3, "point": 4}
OPS = {"const": 0, "var": 1, "add": 2, "sub": 3, "mul": 4, "div": 5, "sqrt": 6, "log": 7,
       "exp": 8, "sin": 9, "cos": 10, "tan": 11, "abs": 12, "neg": 13, "inv": 14, "sq": 15,
       "cube": 16, "cbrt": 17, "tanh": 18, "atan": 19, "sinh": 20, "cosh": 21, "max": 22,
       "min": 23}


def make_mut_params(p_crossover=0.7, p_subtree=0.1, p_hoist=0.05, p_point=0.1,
                    p_replace=0.1, subtree_depth=4, functions=None) -> MutParams:
    names = functions if functions is not None else [n for n, c in OPS.items() if c >= 2]
    mask = 0
    for n in names:
        mask |= 1 << OPS[n]
    m = MutParams()
    m.p_crossover, m.p_subtree, m.p_hoist, m.p_point = p_crossover, p_subtree, p_hoist, p_point
    m.p_point_replace, m.subtree_depth, m.functions = p_replace, subtree_depth, mask
    return m


class EvalOpts(C.Structure):
    _fields_ = [("rows_per_thread", C.c_int), ("chunk_rows", C.c_int),
                ("blocks_per_sm", C.c_int), ("accum", C.c_int),
                ("long_edge", C.c_int), ("long_rows_per_thread", C.c_int),
                ("long_blocks_per_sm", C.c_int), ("reserved", C.c_int * 1)]


def _load():
    # GP_LIBGP selects another build of the same ABI (e.g. an instrumented one)
    path = os.environ.get("GP_LIBGP") or _build.LIB
    if path == _build.LIB and (not os.path.exists(path) or os.environ.get("GP_REBUILD")):
        _build.build()
    if not os.path.exists(path):
        raise ImportError(f"libgp.so missing at {path}; run paper_2110_11226_gb300/build.py")
    lib = C.CDLL(path)
    P, i32, i64, f32, u64 = C.c_void_p, C.c_int, C.c_int64, C.c_float, C.c_uint64
    sig = {
        "gp_version": (C.c_char_p, []),
        "gp_status_string": (C.c_char_p, [i32]),
        "gp_evaluate": (i32, [P, P, i32, P, i64, i32, P, P, i32, P, P]),
        "gp_evaluate_ex": (i32, [P, P, i32, P, i64, i32, P, P, i32, P, P, P, P, P,
                                 C.c_size_t, P]),
        "gp_workspace_size": (C.c_size_t, [i32, i64, i32, P]),
        "gp_resolve_opts": (i32, [i32, i64, i32, P, P]),
        "gp_evaluate_plain": (i32, [P, P, i32, P, i64, i32, P, P, i32, P, P]),
        "gp_predict": (i32, [P, P, i32, P, i64, i32, P, P]),
        "gp_predict_ex": (i32, [P, P, i32, P, i64, i32, P, P, P]),
        "gp_evaluate_host": (i32, [P, P, i32, P, i64, i32, P, P, i32, P, P]),
        "gp_validate_host": (i32, [P, P, i32, i32, P, P]),
        "gp_tournament_ex": (i32, [P, P, i32, i32, i32, f32, i32, u64, u64, P, P]),
        "gp_tournament": (i32, [P, i32, i32, u64, P]),
        "gp_const_grad": (i32, [P, P, i32, P, i64, i32, P, P, i32, P, P, P]),
        "gp_adam_step": (i32, [P, P, i32, P, P, P, i32, f32, f32, f32, f32, P]),
        "gp_get_consts": (i32, [P, P, i32, P, P]),
        "gp_mutate_workspace_size": (C.c_size_t, [i32]),
        "gp_mutate": (i32, [P, P, i32, i32, P, i32, P, u64, u64, P, P, P, P, C.c_size_t, P]),
        "gp_set_consts": (i32, [P, P, i32, P, P]),
        "gp_last_device_status": (i32, [P, P]),
        "gp_autotune": (i32, [P, P, i32, P, i64, i32, P, P, i32, P, P]),
        "gp_probe_pipes": (i32, [P, P]),
        "gp_evaluate_static": (i32, [P, P, i32, P, i64, i32, P, P, i32, P, P]),
        "gp_static_opts": (i32, [i32, i64, i32, i32, P]),
        "gp_timing_enable": (i32, [i32]),
        "gp_timing_read": (i32, [P, P]),
        "gp_shutdown": (None, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()
LIB_PATH = os.environ.get("GP_LIBGP") or _build.LIB


# ---- marshalling helpers -------------------------------------------------
def _on_device(t: torch.Tensor) -> bool:
    return t.is_cuda


def _dptr(t: Optional[torch.Tensor], name: str, dtype=None, numel: Optional[int] = None):
    """Device pointer of `t` (None stays None).  The library reads and writes
    through raw pointers, so the element type and a minimum element count
    are checked here, before anything reaches the GPU."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, not {t.dtype}")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements, the call needs {numel}")
    if not _on_device(t):
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


_F32, _F64, _I32, _I64 = torch.float32, torch.float64, torch.int32, torch.int64


def _progs(progs, offsets):
    """(progs, offsets) pointers: 8-byte node records held as int64, int32
    offsets [n_progs + 1]."""
    return _dptr(progs, "progs", _I64), _dptr(offsets, "offsets", _I32)


def _data(X, y, w, n_rows):
    """(X, y, w) pointers: float32 columns, y and w at least n_rows long."""
    return (_dptr(X, "X", _F32), _dptr(y, "y", _F32, n_rows), _dptr(w, "w", _F32, n_rows))


def _hptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _metric(m):
    return METRICS[m] if isinstance(m, str) else int(m)


def _check(name, rc):
    if rc != 0:
        raise GPError(name, rc)


def _xshape(X):
    if X.dim() != 2:
        raise ValueError("X must be [n_feat][n_rows] (column-major data)")
    return int(X.shape[1]), int(X.shape[0])


def nodes_to_device(nodes: np.ndarray, device="cuda") -> torch.Tensor:
    """numpy node array -> CUDA int64 tensor with the same 8-byte records."""
    n = np.ascontiguousarray(nodes, dtype=NODE_DTYPE)
    return torch.from_numpy(n.view(np.int64).copy()).to(device)


def nodes_from_device(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().view(NODE_DTYPE).copy()


def _nprogs(offsets):
    return int(offsets.numel()) - 1


# ---- entry points --------------------------------------------------------
def gp_version() -> str:
    return _lib.gp_version().decode()


def gp_evaluate(progs, offsets, X, y, w=None, metric="mse", out=None, stream=None):
    n_rows, n_feat = _xshape(X)
    P = _nprogs(offsets)
    if out is None:
        out = torch.empty(P, dtype=torch.float32, device=X.device)
    pp, po = _progs(progs, offsets)
    xp, yp, wp = _data(X, y, w, n_rows)
    _check("gp_evaluate", _lib.gp_evaluate(
        pp, po, P, xp, n_rows, n_feat, yp, wp, _metric(metric),
        _dptr(out, "out", _F32, P), _stream(stream)))
    return out


def gp_evaluate_static(progs, offsets, X, y, w=None, metric="mse", out=None, stream=None):
    """gp_evaluate without any device allocation: the library's fixed
    scratch array serves as workspace (see include/gp.h)."""
    n_rows, n_feat = _xshape(X)
    P = _nprogs(offsets)
    if out is None:
        out = torch.empty(P, dtype=torch.float32, device=X.device)
    pp, po = _progs(progs, offsets)
    xp, yp, wp = _data(X, y, w, n_rows)
    _check("gp_evaluate_static", _lib.gp_evaluate_static(
        pp, po, P, xp, n_rows, n_feat, yp, wp, _metric(metric),
        _dptr(out, "out", _F32, P), _stream(stream)))
    return out


def make_opts(rows_per_thread=0, chunk_rows=0, blocks_per_sm=0, accum="fp64", long_edge=0,
              long_rows_per_thread=0, long_blocks_per_sm=0) -> EvalOpts:
    o = EvalOpts()
    o.rows_per_thread = rows_per_thread
    o.chunk_rows = chunk_rows
    o.blocks_per_sm = blocks_per_sm
    o.accum = ACCUM[accum] if isinstance(accum, str) else int(accum)
    o.long_edge = long_edge
    o.long_rows_per_thread = long_rows_per_thread
    o.long_blocks_per_sm = long_blocks_per_sm
    return o


def gp_evaluate_ex(progs, offsets, X, y, w=None, metric="mse", opts: Optional[EvalOpts] = None,
                   out=None, out64=None, out_status=None, ws=None, stream=None):
    n_rows, n_feat = _xshape(X)
    P = _nprogs(offsets)
    if out is None:
        out = torch.empty(P, dtype=torch.float32, device=X.device)
    ws_ptr, ws_bytes = (None, 0) if ws is None else (_dptr(ws, "ws"), ws.numel() * ws.element_size())
    pp, po = _progs(progs, offsets)
    xp, yp, wp = _data(X, y, w, n_rows)
    _check("gp_evaluate_ex", _lib.gp_evaluate_ex(
        pp, po, P, xp, n_rows, n_feat, yp, wp, _metric(metric),
        None if opts is None else C.byref(opts), _dptr(out, "out", _F32, P),
        _dptr(out64, "out64", _F64, P), _dptr(out_status, "out_status", _I32, P), ws_ptr, ws_bytes,
        _stream(stream)))
    return out


def gp_workspace_size(n_progs, n_rows, n_feat, opts: Optional[EvalOpts] = None) -> int:
    return int(_lib.gp_workspace_size(int(n_progs), int(n_rows), int(n_feat),
                                      None if opts is None else C.byref(opts)))


def gp_resolve_opts(n_progs, n_rows, n_feat, opts: Optional[EvalOpts] = None) -> EvalOpts:
    out = EvalOpts()
    _check("gp_resolve_opts", _lib.gp_resolve_opts(int(n_progs), int(n_rows), int(n_feat),
                                                   None if opts is None else C.byref(opts),
                                                   C.byref(out)))
    return out


def gp_static_opts(n_progs, n_rows, n_feat, metric="mse") -> EvalOpts:
    """The tunables gp_evaluate_static uses for this problem."""
    out = EvalOpts()
    _check("gp_static_opts", _lib.gp_static_opts(int(n_progs), int(n_rows), int(n_feat),
                                                 _metric(metric), C.byref(out)))
    return out


def gp_evaluate_plain(progs, offsets, X, y, w=None, metric="mse", out=None, stream=None):
    n_rows, n_feat = _xshape(X)
    P = _nprogs(offsets)
    if out is None:
        out = torch.empty(P, dtype=torch.float32, device=X.device)
    pp, po = _progs(progs, offsets)
    xp, yp, wp = _data(X, y, w, n_rows)
    _check("gp_evaluate_plain", _lib.gp_evaluate_plain(
        pp, po, P, xp, n_rows, n_feat, yp, wp, _metric(metric),
        _dptr(out, "out", _F32, P), _stream(stream)))
    return out


def gp_predict(progs, offsets, X, out=None, stream=None):
    n_rows, n_feat = _xshape(X)
    P = _nprogs(offsets)
    if out is None:
        out = torch.empty((P, n_rows), dtype=torch.float32, device=X.device)
    pp, po = _progs(progs, offsets)
    _check("gp_predict", _lib.gp_predict(
        pp, po, P, _dptr(X, "X", _F32), n_rows, n_feat, _dptr(out, "out", _F32, P * n_rows),
        _stream(stream)))
    return out


def gp_predict_ex(progs, offsets, X, opts: Optional[EvalOpts] = None, out=None, stream=None):
    n_rows, n_feat = _xshape(X)
    P = _nprogs(offsets)
    if out is None:
        out = torch.empty((P, n_rows), dtype=torch.float32, device=X.device)
    pp, po = _progs(progs, offsets)
    _check("gp_predict_ex", _lib.gp_predict_ex(
        pp, po, P, _dptr(X, "X", _F32), n_rows, n_feat, None if opts is None else C.byref(opts),
        _dptr(out, "out", _F32, P * n_rows), _stream(stream)))
    return out


def gp_evaluate_host(nodes: np.ndarray, offsets: np.ndarray, X: np.ndarray, y: np.ndarray,
                     w: Optional[np.ndarray] = None, metric="mse", out: Optional[np.ndarray] = None,
                     stream=None) -> np.ndarray:
    """Host arrays in, host fitness out (copies inside the call, synchronous)."""
    nodes = np.ascontiguousarray(nodes, dtype=NODE_DTYPE)
    offsets = np.ascontiguousarray(offsets, dtype=np.int32)
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    w = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
    P = len(offsets) - 1
    if out is None:
        out = np.empty(P, np.float32)
    _check("gp_evaluate_host", _lib.gp_evaluate_host(
        _hptr(nodes), _hptr(offsets), P, _hptr(X), X.shape[1], X.shape[0], _hptr(y), _hptr(w),
        _metric(metric), _hptr(out), _stream(stream)))
    return out


def gp_validate_host(nodes: np.ndarray, offsets: np.ndarray, n_feat: int):
    """Returns (rc, status[P], high_water[P]) -- runs on the host, no GPU needed."""
    nodes = np.ascontiguousarray(nodes, dtype=NODE_DTYPE)
    offsets = np.ascontiguousarray(offsets, dtype=np.int32)
    P = len(offsets) - 1
    st = np.zeros(P, np.int32)
    hw = np.zeros(P, np.int32)
    rc = _lib.gp_validate_host(_hptr(nodes), _hptr(offsets), P, int(n_feat), _hptr(st), _hptr(hw))
    return int(rc), st, hw


def gp_tournament_ex(fitness, n_tourn, tourn_size, seed, offsets=None, parsimony=0.0,
                     greater_is_better=False, offset=0, out=None, stream=None):
    P = int(fitness.numel())
    if out is None:
        out = torch.empty(n_tourn, dtype=torch.int32, device=fitness.device)
    _check("gp_tournament_ex", _lib.gp_tournament_ex(
        _dptr(fitness, "fitness", _F32), _dptr(offsets, "offsets", _I32, P + 1), P, int(n_tourn),
        int(tourn_size), float(parsimony), int(bool(greater_is_better)), int(seed), int(offset),
        _dptr(out, "out", _I32, int(n_tourn)), _stream(stream)))
    return out


def gp_tournament(fitness, tourn_size, seed, out=None):
    P = int(fitness.numel())
    if out is None:
        out = torch.empty(P, dtype=torch.int32, device=fitness.device)
    _check("gp_tournament", _lib.gp_tournament(
        _dptr(fitness, "fitness", _F32), P, int(tourn_size), int(seed), _dptr(out, "out", _I32, P)))
    return out


def gp_const_grad(progs, offsets, X, y, w=None, metric="mse", out_grad=None, out_fitness=None,
                  stream=None):
    n_rows, n_feat = _xshape(X)
    P = _nprogs(offsets)
    if out_grad is None:
        out_grad = torch.empty((P, MAX_CONSTS), dtype=torch.float32, device=X.device)
    if out_fitness is None:
        out_fitness = torch.empty(P, dtype=torch.float32, device=X.device)
    pp, po = _progs(progs, offsets)
    xp, yp, wp = _data(X, y, w, n_rows)
    _check("gp_const_grad", _lib.gp_const_grad(
        pp, po, P, xp, n_rows, n_feat, yp, wp, _metric(metric),
        _dptr(out_grad, "out_grad", _F32, P * MAX_CONSTS),
        _dptr(out_fitness, "out_fitness", _F32, P), _stream(stream)))
    return out_grad, out_fitness


def gp_adam_step(progs, offsets, grad, m, v, step, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8,
                 stream=None):
    P = _nprogs(offsets)
    n = P * MAX_CONSTS
    _check("gp_adam_step", _lib.gp_adam_step(
        *_progs(progs, offsets), P, _dptr(grad, "grad", _F32, n), _dptr(m, "m", _F32, n),
        _dptr(v, "v", _F32, n), int(step), float(lr), float(beta1), float(beta2), float(eps),
        _stream(stream)))


def gp_get_consts(progs, offsets, out=None, stream=None):
    P = _nprogs(offsets)
    if out is None:
        out = torch.empty((P, MAX_CONSTS), dtype=torch.float32, device=progs.device)
    _check("gp_get_consts", _lib.gp_get_consts(*_progs(progs, offsets), P,
                                               _dptr(out, "out", _F32, P * MAX_CONSTS),
                                               _stream(stream)))
    return out


def gp_set_consts(progs, offsets, consts, stream=None):
    P = _nprogs(offsets)
    if consts.shape != (P, MAX_CONSTS) or consts.dtype != torch.float32:
        raise GPError(f"gp_set_consts: consts must be float32 [{P}, {MAX_CONSTS}]")
    _check("gp_set_consts", _lib.gp_set_consts(*_progs(progs, offsets), P,
                                               _dptr(consts, "consts"), _stream(stream)))


class ConstantsFitness(torch.autograd.Function):
    """fitness[P] as a differentiable function of the constants [P, 16].

    forward writes the constants into the programs' nodes (in place, like
    gp_adam_step) and runs gp_const_grad, which returns the fitness and its
    gradient in one pass; backward scales that gradient by the incoming one.
    Slots past a program's constant count get gradient 0."""

    @staticmethod
    def forward(ctx, consts, progs, offsets, X, y, w, metric):
        c = consts.detach().contiguous()
        gp_set_consts(progs, offsets, c)
        grad, fit = gp_const_grad(progs, offsets, X, y, w, metric)
        ctx.save_for_backward(grad)
        return fit

    @staticmethod
    def backward(ctx, g_fit):
        (grad,) = ctx.saved_tensors
        return grad * g_fit.unsqueeze(1), None, None, None, None, None, None


def fitness_of_constants(consts, progs, offsets, X, y, w=None, metric="mse"):
    return ConstantsFitness.apply(consts, progs, offsets, X, y, w, metric)


def gp_mutate(progs, offsets, n_feat, parents, params: Optional[MutParams] = None, seed=0,
              offset=0, out=None, out_offsets=None, out_kind=None, ws=None, stream=None):
    """Next population on the device; returns (nodes, offsets, kind) tensors.
    `nodes` has capacity n_out * 255; its first offsets[-1] entries are used."""
    P = _nprogs(offsets)
    n_out = int(parents.numel()) // 2
    dev = progs.device
    if params is None:
        params = make_mut_params()
    if out is None:
        out = torch.empty(n_out * 255, dtype=torch.int64, device=dev)
    if out_offsets is None:
        out_offsets = torch.empty(n_out + 1, dtype=torch.int32, device=dev)
    if out_kind is None:
        out_kind = torch.empty(n_out, dtype=torch.int32, device=dev)
    ws_bytes = 0 if ws is None else ws.numel() * ws.element_size()
    _check("gp_mutate", _lib.gp_mutate(
        *_progs(progs, offsets), P, int(n_feat), _dptr(parents, "parents", _I32), n_out,
        C.byref(params), int(seed), int(offset), _dptr(out, "out", _I64, n_out * 255),
        _dptr(out_offsets, "out_offsets", _I32, n_out + 1),
        _dptr(out_kind, "out_kind", _I32, n_out), _dptr(ws, "ws"), ws_bytes, _stream(stream)))
    return out, out_offsets, out_kind


def gp_mutate_workspace_size(n_out) -> int:
    return int(_lib.gp_mutate_workspace_size(int(n_out)))


def gp_last_device_status(stream=None) -> int:
    flags = C.c_uint32(0)
    _check("gp_last_device_status", _lib.gp_last_device_status(_stream(stream), C.byref(flags)))
    return int(flags.value)


def gp_autotune(progs, offsets, X, y, w=None, metric="mse", stream=None) -> EvalOpts:
    n_rows, n_feat = _xshape(X)
    best = EvalOpts()
    pp, po = _progs(progs, offsets)
    xp, yp, wp = _data(X, y, w, n_rows)
    _check("gp_autotune", _lib.gp_autotune(
        pp, po, _nprogs(offsets), xp, n_rows, n_feat, yp, wp, _metric(metric), C.byref(best),
        _stream(stream)))
    return best


def gp_probe_pipes(stream=None) -> dict:
    out = (C.c_double * 8)()
    _check("gp_probe_pipes", _lib.gp_probe_pipes(out, _stream(stream)))
    return {"fp32": out[0], "ex2": out[1], "rcp": out[2], "rsqrt": out[3], "lg2": out[4],
            "sin": out[5], "sms": int(out[6]), "unit": "lane-operations/s"}


def gp_timing_enable(on: bool = True):
    _check("gp_timing_enable", _lib.gp_timing_enable(int(bool(on))))


def gp_timing_read():
    """(total ms, number of evaluations) of the evaluator launches since the last read."""
    ms = C.c_double(0.0)
    n = C.c_int(0)
    _check("gp_timing_read", _lib.gp_timing_read(C.byref(ms), C.byref(n)))
    return float(ms.value), int(n.value)


def gp_shutdown():
    _lib.gp_shutdown()
