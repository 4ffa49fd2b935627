"""CPU oracle for stack-based GP fitness evaluation (arXiv 2110.11226).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the product path never
does.  It shares no code with the CUDA library.

The arithmetic lives in ``gp_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off`` so that its FP32 mode rounds every operation the way
IEEE single precision does).  This module only builds it with gcc and
marshals numpy arrays.  Sections cited per function are the paper's.

Parity pins for every function are in ``tests/test_oracle_pins.py``; none of
them is "parity unpinned" except where that file says so.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
# A test that plants mistakes in a copy of the oracle points this at the copy.
_SO_OVERRIDE = os.environ.get("GP_ORACLE_SO")
_lock = threading.Lock()
_lib = None

# Layout of one program node: int16 op, int16 feat, float32 c (8 bytes).
NODE_DTYPE = np.dtype([("op", "<i2"), ("feat", "<i2"), ("c", "<f4")])

# Op numbering of the input format, written out here on its own.
OPS = {
    "const": 0, "var": 1, "add": 2, "sub": 3, "mul": 4, "div": 5,
    "sqrt": 6, "log": 7, "exp": 8, "sin": 9, "cos": 10, "tan": 11,
    "abs": 12, "neg": 13, "inv": 14, "sq": 15, "cube": 16, "cbrt": 17,
    "tanh": 18, "atan": 19, "sinh": 20, "cosh": 21, "max": 22, "min": 23,
}
METRICS = {"mae": 0, "mse": 1, "rmse": 2, "logloss": 3, "pearson": 4, "spearman": 5}
MAX_STACK = 20
MAX_LEN = 255
MAX_CONSTS = 16
THRESHOLD = np.float32(0.001)

# Status codes of validate().
OK, BAD_LENGTH, BAD_OP, BAD_FEATURE, UNDERFLOW, LEFTOVER, TOO_DEEP = range(7)


def build(force: bool = False) -> str:
    """Compile gp_oracle.c into a shared library (gcc, OpenMP)."""
    with _lock:
        if (not force and os.path.exists(_SO)
                and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
            return _SO
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-Wall",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
        return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if _SO_OVERRIDE:
        lib = C.CDLL(_SO_OVERRIDE)
    else:
        build()
        lib = C.CDLL(_SO)
    P = C.c_void_p
    i64, i32, f64 = C.c_int64, C.c_int, C.c_double
    lib.ora_op_name.restype = C.c_char_p
    lib.ora_op_name.argtypes = [i32]
    lib.ora_op_arity.argtypes = [i32]
    lib.ora_validate.argtypes = [P, i32, i32, P]
    lib.ora_predict64.argtypes = [P, P, i32, P, i64, i64, i64, P, P, i32]
    lib.ora_predict32.argtypes = [P, P, i32, P, i64, i64, i64, P, i32]
    lib.ora_predict_bound.argtypes = [P, P, i32, P, i64, i64, i64, f64,
                                      P, P, P, i32]
    lib.ora_loss.restype = f64
    lib.ora_loss.argtypes = [i32, f64, f64]
    lib.ora_fitness.argtypes = [P, P, i32, P, i64, P, P, i32, i64, i64,
                                P, P, i32]
    lib.ora_philox4x32_10.argtypes = [P, P, P]
    lib.ora_tournament_draw.restype = i64
    lib.ora_tournament_draw.argtypes = [C.c_uint64, C.c_uint64, i64, i32, i32]
    lib.ora_tournament.argtypes = [P, P, i32, i64, i32, C.c_float, i32,
                                   C.c_uint64, C.c_uint64, P]
    lib.ora_count_consts.argtypes = [P, i32]
    lib.ora_const_grad.argtypes = [P, P, i32, P, i64, P, P, i32, i64, i64,
                                   P, P, P, i32]
    lib.ora_const_grad32.argtypes = [P, P, i32, P, i64, P, P, i32, i64, i64,
                                     P, P, i32]
    lib.ora_adam.argtypes = [P, P, P, P, i64, i32, f64, f64, f64, f64]
    lib.ora_average_ranks.argtypes = [P, i64, P]
    lib.ora_spearman_of.restype = f64
    lib.ora_spearman_of.argtypes = [P, P, P, i64]
    lib.ora_mutate.argtypes = [P, P, i32, i32, P, i32, P, i32, C.c_uint32, C.c_uint64,
                               C.c_uint64, P, P, P]
    lib.ora_max_threads.restype = i32
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _progs(progs, offsets):
    progs = np.ascontiguousarray(progs, dtype=NODE_DTYPE)
    offsets = np.ascontiguousarray(offsets, dtype=np.int32)
    return progs, offsets


def _colmajor(X):
    """X as float32 [n_feat][n_rows] (column-major data, one row per feature)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    assert X.ndim == 2
    return X


def op_name(op: int) -> str:
    return _load().ora_op_name(int(op)).decode()


def op_arity(op: int) -> int:
    return int(_load().ora_op_arity(int(op)))


def max_threads() -> int:
    return int(_load().ora_max_threads())


def validate(prog, n_feat: int):
    """Sec. III-C2: a stack of 20 evaluates the program.  Returns (status, high_water)."""
    prog = np.ascontiguousarray(prog, dtype=NODE_DTYPE)
    hw = np.zeros(1, np.int32)
    s = _load().ora_validate(_ptr(prog), len(prog), int(n_feat), _ptr(hw))
    return int(s), int(hw[0])


def predict64(progs, offsets, X, row0=0, n_eval=None, n_threads=0):
    """FP64 value of every program on every row (Sec. III-A reverse scan).

    Returns (pred [P, n_eval] float64, status [P] int32)."""
    lib = _load()
    progs, offsets = _progs(progs, offsets)
    X = _colmajor(X)
    n_rows = X.shape[1]
    n_eval = n_rows - row0 if n_eval is None else n_eval
    P = len(offsets) - 1
    out = np.empty((P, n_eval), np.float64)
    st = np.zeros(P, np.int32)
    lib.ora_predict64(_ptr(progs), _ptr(offsets), P, _ptr(X), n_rows, row0,
                      n_eval, _ptr(out), _ptr(st), n_threads)
    return out, st


def predict32(progs, offsets, X, row0=0, n_eval=None, n_threads=0):
    """Same scan with every operation rounded to float (C library float functions)."""
    lib = _load()
    progs, offsets = _progs(progs, offsets)
    X = _colmajor(X)
    n_rows = X.shape[1]
    n_eval = n_rows - row0 if n_eval is None else n_eval
    P = len(offsets) - 1
    out = np.empty((P, n_eval), np.float32)
    lib.ora_predict32(_ptr(progs), _ptr(offsets), P, _ptr(X), n_rows, row0,
                      n_eval, _ptr(out), n_threads)
    return out


def predict_bound(progs, offsets, X, row0=0, n_eval=None, ulps_fn=4.0,
                  n_threads=0):
    """FP64 values, a first-order bound on the error of an FP32 evaluation
    and per-row flags (1 = protected-operator decision may flip, 2 = out of
    float range or bound meaningless)."""
    lib = _load()
    progs, offsets = _progs(progs, offsets)
    X = _colmajor(X)
    n_rows = X.shape[1]
    n_eval = n_rows - row0 if n_eval is None else n_eval
    P = len(offsets) - 1
    v = np.empty((P, n_eval), np.float64)
    e = np.empty((P, n_eval), np.float64)
    fl = np.empty((P, n_eval), np.uint8)
    lib.ora_predict_bound(_ptr(progs), _ptr(offsets), P, _ptr(X), n_rows,
                          row0, n_eval, float(ulps_fn), _ptr(v), _ptr(e),
                          _ptr(fl), n_threads)
    return v, e, fl


def loss(metric, p, y) -> float:
    m = METRICS[metric] if isinstance(metric, str) else int(metric)
    return float(_load().ora_loss(m, float(p), float(y)))


def fitness(progs, offsets, X, y, w=None, metric="mse", row0=0, n_eval=None,
            n_threads=0):
    """Weighted fitness per program (Sec. III-C3).  Returns (fit [P], status [P])."""
    lib = _load()
    progs, offsets = _progs(progs, offsets)
    X = _colmajor(X)
    y = np.ascontiguousarray(y, np.float32)
    w = None if w is None else np.ascontiguousarray(w, np.float32)
    n_rows = X.shape[1]
    n_eval = n_rows - row0 if n_eval is None else n_eval
    P = len(offsets) - 1
    m = METRICS[metric] if isinstance(metric, str) else int(metric)
    out = np.empty(P, np.float64)
    st = np.zeros(P, np.int32)
    rc = lib.ora_fitness(_ptr(progs), _ptr(offsets), P, _ptr(X), n_rows,
                         _ptr(y), _ptr(w), m, row0, n_eval, _ptr(out),
                         _ptr(st), n_threads)
    if rc != 0:
        raise ValueError("oracle fitness: bad metric or zero total weight")
    return out, st


def philox4x32_10(ctr, key):
    """Philox4x32-10 (Salmon et al. 2011) on one counter / key."""
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    o = np.empty(4, np.uint32)
    _load().ora_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def tournament_draw(seed, offset, t, j, n_progs) -> int:
    return int(_load().ora_tournament_draw(int(seed), int(offset), int(t),
                                           int(j), int(n_progs)))


def tournament(fitness_, n_tourn, k, seed, lengths=None, parsimony=0.0,
               greater_is_better=False, offset=0):
    """Sec. III-C1 tournament selection; returns winners [n_tourn] int32."""
    f = np.ascontiguousarray(fitness_, np.float32)
    ln = None if lengths is None else np.ascontiguousarray(lengths, np.int32)
    out = np.empty(n_tourn, np.int32)
    rc = _load().ora_tournament(_ptr(f), _ptr(ln), len(f), int(n_tourn),
                                int(k), float(parsimony),
                                int(bool(greater_is_better)), int(seed),
                                int(offset), _ptr(out))
    if rc != 0:
        raise ValueError("oracle tournament: bad arguments")
    return out


def count_consts(prog) -> int:
    prog = np.ascontiguousarray(prog, dtype=NODE_DTYPE)
    return int(_load().ora_count_consts(_ptr(prog), len(prog)))


def const_grad(progs, offsets, X, y, w=None, metric="mse", row0=0,
               n_eval=None, n_threads=0, with_abs=False):
    """Reverse-mode gradient of fitness w.r.t. each program's constants
    (constant k = k-th CONST node in prefix order).  Returns (grad [P,16],
    fit [P]), plus gabs [P,16] (the same sums of absolute per-row
    contributions) when with_abs."""
    lib = _load()
    progs, offsets = _progs(progs, offsets)
    X = _colmajor(X)
    y = np.ascontiguousarray(y, np.float32)
    w = None if w is None else np.ascontiguousarray(w, np.float32)
    n_rows = X.shape[1]
    n_eval = n_rows - row0 if n_eval is None else n_eval
    P = len(offsets) - 1
    m = METRICS[metric] if isinstance(metric, str) else int(metric)
    g = np.empty((P, MAX_CONSTS), np.float64)
    f = np.empty(P, np.float64)
    ga = np.empty((P, MAX_CONSTS), np.float64) if with_abs else None
    rc = lib.ora_const_grad(_ptr(progs), _ptr(offsets), P, _ptr(X), n_rows,
                            _ptr(y), _ptr(w), m, row0, n_eval, _ptr(g),
                            _ptr(f), _ptr(ga), n_threads)
    if rc == -1:
        raise ValueError("oracle const_grad: bad metric or zero total weight")
    return (g, f, ga) if with_abs else (g, f)


def const_grad32(progs, offsets, X, y, w=None, metric="mse", row0=0,
                 n_eval=None, n_threads=0):
    """The reverse mode with every per-row operation in FP32 (sums over rows
    in FP64): how far FP32 rounding alone moves each gradient.  Returns
    (grad [P,16], fit [P])."""
    lib = _load()
    progs, offsets = _progs(progs, offsets)
    X = _colmajor(X)
    y = np.ascontiguousarray(y, np.float32)
    w = None if w is None else np.ascontiguousarray(w, np.float32)
    n_rows = X.shape[1]
    n_eval = n_rows - row0 if n_eval is None else n_eval
    P = len(offsets) - 1
    m = METRICS[metric] if isinstance(metric, str) else int(metric)
    g = np.empty((P, MAX_CONSTS), np.float64)
    f = np.empty(P, np.float64)
    rc = lib.ora_const_grad32(_ptr(progs), _ptr(offsets), P, _ptr(X), n_rows,
                              _ptr(y), _ptr(w), m, row0, n_eval, _ptr(g),
                              _ptr(f), n_threads)
    if rc == -1:
        raise ValueError("oracle const_grad32: bad metric or zero total weight")
    return g, f


def adam(theta, g, m, v, step, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) in FP64, in place on theta, m, v."""
    for a in (theta, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = np.ascontiguousarray(g, np.float64)
    _load().ora_adam(_ptr(theta), _ptr(g), _ptr(m), _ptr(v), theta.size,
                     int(step), float(lr), float(beta1), float(beta2),
                     float(eps))


MUT_KINDS = {"reproduction": 0, "crossover": 1, "subtree": 2, "hoist": 3, "point": 4}


def mutate(progs, offsets, n_feat, parents, p_crossover=0.7, p_subtree=0.1, p_hoist=0.05,
           p_point=0.1, p_replace=0.1, subtree_depth=4, functions=None, seed=0, offset=0):
    """One offspring per pair (parents[2t], parents[2t+1]) (Sec. II-A mutation
    kinds, Sec. III-C2 hoisted crossover).  functions: op names new function
    nodes may take (default: every function).  Returns (nodes, offsets, kind)."""
    lib = _load()
    progs, offsets = _progs(progs, offsets)
    parents = np.ascontiguousarray(parents, np.int32)
    n_out = len(parents) // 2
    names = functions if functions is not None else [n for n, c in OPS.items() if c >= 2]
    mask = 0
    for n in names:
        mask |= 1 << OPS[n]
    # the probabilities are float32 values, as the library takes them
    probs = np.array([p_crossover, p_subtree, p_hoist, p_point, p_replace],
                     np.float32).astype(np.float64)
    out = np.zeros(max(1, n_out) * 255, NODE_DTYPE)
    off = np.zeros(n_out + 1, np.int32)
    kind = np.zeros(max(1, n_out), np.int32)
    rc = lib.ora_mutate(_ptr(progs), _ptr(offsets), len(offsets) - 1, int(n_feat), _ptr(parents),
                        n_out, _ptr(probs), int(subtree_depth), mask, int(seed), int(offset),
                        _ptr(out), _ptr(off), _ptr(kind))
    if rc != 0:
        raise ValueError("oracle mutate: bad arguments")
    return out[:off[-1]].copy(), off, kind[:n_out].copy()


def average_ranks(v):
    """1-based ranks of v, ties sharing the mean of their positions."""
    v = np.ascontiguousarray(v, np.float64)
    out = np.empty(len(v), np.float64)
    if _load().ora_average_ranks(_ptr(v), len(v), _ptr(out)) != 0:
        raise ValueError("NaN in ranked values")
    return out


def spearman_of(pred, y, w=None) -> float:
    """Spearman fitness |r_s| of given predictions (Sec. III-C3)."""
    p = np.ascontiguousarray(pred, np.float64)
    y = np.ascontiguousarray(y, np.float32)
    w = None if w is None else np.ascontiguousarray(w, np.float32)
    return float(_load().ora_spearman_of(_ptr(p), _ptr(y), _ptr(w), len(p)))

