"""Seeded synthetic inputs: datasets and random program populations.

This module is shared by the tests, the benchmark and the oracle checks.  It
holds none of the evaluation arithmetic (no prefix-list evaluator, no
protected operators, no loss): it only draws data and program trees.

Layouts (the library's input format):
  * X: float32, column-major, shape [n_feat][n_rows] (one contiguous column
    per feature), as the paper keeps its training data (Sec. III).
  * programs: one flat array of 8-byte nodes (int16 op, int16 feat,
    float32 c) in prefix order, plus int32 offsets[P+1] (Sec. III-A).

Workloads (stand-ins for the paper's datasets, which are not available):
  * Pagie-1 (Sec. IV-A, Eq. pagie): x0, x1 ~ U[-5, 5] i.i.d.
  * Large tabular regression shaped like Higgs (11M x 28, Sec. IV-B).
  * Binary classification with class weights.
The hidden target programs of the tabular and classification workloads draw
their functions from {add, sub, mul, sin, cos, abs, neg}, which need no
protection, and are composed directly on numpy arrays.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence, Tuple

import numpy as np

NODE_DTYPE = np.dtype([("op", "<i2"), ("feat", "<i2"), ("c", "<f4")])

# Op numbering of the input format and the arity of each op.
OP = {
    "const": 0, "var": 1, "add": 2, "sub": 3, "mul": 4, "div": 5,
    "sqrt": 6, "log": 7, "exp": 8, "sin": 9, "cos": 10, "tan": 11,
    "abs": 12, "neg": 13, "inv": 14, "sq": 15, "cube": 16, "cbrt": 17,
    "tanh": 18, "atan": 19, "sinh": 20, "cosh": 21, "max": 22, "min": 23,
}
ARITY = {0: 0, 1: 0, 2: 2, 3: 2, 4: 2, 5: 2, 6: 1, 7: 1, 8: 1, 9: 1,
         10: 1, 11: 1, 12: 1, 13: 1, 14: 1, 15: 1, 16: 1, 17: 1, 18: 1,
         19: 1, 20: 1, 21: 1, 22: 2, 23: 2}
OP_NAME = {v: k for k, v in OP.items()}

BASIC_SET = ("add", "sub", "mul", "div")
FULL_SET = ("add", "sub", "mul", "div", "sqrt", "log", "exp", "sin", "cos",
            "abs", "neg", "inv")
PAPER_SET = ("add", "sub", "mul", "div", "sin", "cos", "tan")
EXTENDED_SET = FULL_SET + ("tan", "sq", "cube", "cbrt", "tanh", "atan", "sinh", "cosh",
                           "max", "min")
SAFE_SET = ("add", "sub", "mul", "sin", "cos", "abs", "neg")

MAX_LEN = 255
MAX_STACK = 20


# --------------------------------------------------------------------------
# trees
# --------------------------------------------------------------------------
def _grow_tree(rng, depth, method, funcs, n_feat, const_range, out):
    """Append one random tree in prefix order to `out` (list of tuples).

    depth = edges left to the deepest allowed terminal.  A grow node below
    the depth limit is a terminal with probability T / (T + F), with T = 2
    terminal kinds (variable, constant) and F = len(funcs)."""
    n_f = len(funcs)
    is_term = depth == 0 or (method == "grow" and rng.random() < 2.0 / (2.0 + n_f))
    if is_term:
        if rng.random() < n_feat / (n_feat + 1.0):
            out.append((OP["var"], int(rng.integers(n_feat)), 0.0))
        else:
            out.append((OP["const"], 0, float(rng.uniform(*const_range))))
        return
    name = funcs[int(rng.integers(n_f))]
    op = OP[name]
    out.append((op, 0, 0.0))
    for _ in range(ARITY[op]):
        _grow_tree(rng, depth - 1, method, funcs, n_feat, const_range, out)


def stack_high_water(nodes: Sequence[Tuple[int, int, float]]) -> int:
    """Largest stack height of the reverse scan (Sec. III-A, III-C2)."""
    sp = mx = 0
    for op, _, _ in reversed(nodes):
        a = ARITY[op]
        sp = sp + 1 if a == 0 else sp - a + 1
        mx = max(mx, sp)
    return mx


def tree_depth(nodes: Sequence[Tuple[int, int, float]]) -> int:
    """Edges from the root to the deepest leaf of a prefix list."""
    depth_stack = []  # remaining children at each open level
    best = 0
    for op, _, _ in nodes:
        d = len(depth_stack)
        best = max(best, d)
        a = ARITY[op]
        if a > 0:
            depth_stack.append(a)
        else:
            while depth_stack:
                depth_stack[-1] -= 1
                if depth_stack[-1] > 0:
                    break
                depth_stack.pop()
    return best


def pack(programs: List[List[Tuple[int, int, float]]]):
    """Flatten a list of prefix lists into (nodes, offsets)."""
    lens = np.array([len(p) for p in programs], np.int64)
    offsets = np.zeros(len(programs) + 1, np.int32)
    offsets[1:] = np.cumsum(lens)
    nodes = np.zeros(int(offsets[-1]), NODE_DTYPE)
    flat = [n for p in programs for n in p]
    if flat:
        arr = np.array(flat, dtype=[("op", "<i8"), ("feat", "<i8"), ("c", "<f8")])
        nodes["op"] = arr["op"]
        nodes["feat"] = arr["feat"]
        nodes["c"] = arr["c"].astype(np.float32)
    return nodes, offsets


def unpack(nodes, offsets) -> List[List[Tuple[int, int, float]]]:
    out = []
    for p in range(len(offsets) - 1):
        seg = nodes[offsets[p]:offsets[p + 1]]
        out.append([(int(n["op"]), int(n["feat"]), float(n["c"])) for n in seg])
    return out


def ramped_half_and_half(n_progs: int, depth_min: int, depth_max: int,
                         funcs: Sequence[str], n_feat: int, seed: int,
                         max_len: int = MAX_LEN,
                         max_consts: Optional[int] = None,
                         const_range=(-1.0, 1.0)):
    """Ramped half-and-half initialisation (Sec. II-A, after Koza).

    Program i gets depth depth_min + (i mod n_depths) and the full method
    for even (i div n_depths), grow otherwise.  Programs longer than max_len
    nodes (or with more than max_consts constants) are drawn again."""
    rng = np.random.default_rng(seed)
    n_depths = depth_max - depth_min + 1
    programs = []
    for i in range(n_progs):
        d = depth_min + (i % n_depths)
        method = "full" if (i // n_depths) % 2 == 0 else "grow"
        for _attempt in range(10000):
            out: list = []
            _grow_tree(rng, d, method, funcs, n_feat, const_range, out)
            if len(out) > max_len:
                continue
            if max_consts is not None and sum(1 for n in out if n[0] == OP["const"]) > max_consts:
                continue
            break
        else:
            raise RuntimeError("could not draw a program within the length cap")
        programs.append(out)
    return pack(programs)


def random_programs(n_progs: int, depth_max: int, funcs: Sequence[str],
                    n_feat: int, seed: int, max_len: int = MAX_LEN):
    """Grow-method programs of random depth in [0, depth_max] (edge cases:
    single terminals, unary chains, deep spines)."""
    rng = np.random.default_rng(seed)
    programs = []
    for _ in range(n_progs):
        while True:
            out: list = []
            _grow_tree(rng, int(rng.integers(depth_max + 1)), "grow", funcs,
                       n_feat, (-1.0, 1.0), out)
            if len(out) <= max_len:
                break
        programs.append(out)
    return pack(programs)


# --------------------------------------------------------------------------
# datasets
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Dataset:
    X: np.ndarray            # float32 [n_feat][n_rows]
    y: np.ndarray            # float32 [n_rows]
    w: Optional[np.ndarray]  # float32 [n_rows] or None (all ones)
    name: str
    hidden: Optional[Tuple[np.ndarray, np.ndarray]] = None

    @property
    def n_rows(self):
        return self.X.shape[1]

    @property
    def n_feat(self):
        return self.X.shape[0]


def pagie_data(n_rows: int, seed: int) -> Dataset:
    """Pagie-1 (Sec. IV-A, Eq. pagie): y = 1/(1+x0^-4) + 1/(1+x1^-4),
    written as x^4/(1+x^4) so that it is finite at 0; x ~ U[-5, 5]."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(-5.0, 5.0, size=(2, n_rows)).astype(np.float32)
    x = X.astype(np.float64)
    x4 = x ** 4
    y = (x4[0] / (1.0 + x4[0]) + x4[1] / (1.0 + x4[1])).astype(np.float32)
    return Dataset(X, y, None, f"pagie1_n{n_rows}")


def _hidden_program(rng, depth, n_use, exact_depth=True):
    while True:
        out: list = []
        _grow_tree(rng, depth, "grow", SAFE_SET, n_use, (-1.0, 1.0), out)
        if not exact_depth or tree_depth(out) == depth:
            return out


def _compose(nodes, X):
    """Value of a SAFE_SET tree (FP64, numpy), by recursive descent."""
    pos = 0

    def rec():
        nonlocal pos
        op, feat, c = nodes[pos]
        pos += 1
        name = OP_NAME[op]
        if name == "const":
            return np.full(X.shape[1], np.float64(np.float32(c)))
        if name == "var":
            return X[feat].astype(np.float64)
        if ARITY[op] == 1:
            a = rec()
            return {"sin": np.sin, "cos": np.cos, "abs": np.abs,
                    "neg": np.negative}[name](a)
        a = rec()
        b = rec()
        return {"add": np.add, "sub": np.subtract, "mul": np.multiply}[name](a, b)

    return rec()


def tabular_data(n_rows: int, seed: int, n_feat: int = 28,
                 n_heavy: int = 4, n_used: int = 8, depth: int = 6) -> Dataset:
    """Higgs-shaped regression (Sec. IV-B): features N(0,1), the first
    n_heavy Student-t (nu = 3); y = hidden depth-6 program over the first
    n_used features + N(0, (0.1 std h)^2)."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n_feat, n_rows), dtype=np.float32)
    X[:n_heavy] = rng.standard_t(3.0, size=(n_heavy, n_rows)).astype(np.float32)
    hid = _hidden_program(rng, depth, n_used)
    h = _compose(hid, X)
    sd = float(np.std(h)) if n_rows > 1 else 0.0
    y = (h + rng.normal(0.0, 0.1 * sd if sd > 0 else 0.0, size=n_rows)).astype(np.float32)
    return Dataset(X, y, None, f"tabular_n{n_rows}_f{n_feat}", pack([hid]))


def classification_data(n_rows: int, seed: int, n_feat: int = 50,
                        depth: int = 5, flip: float = 0.05,
                        w_pos: float = 1.0, w_neg: float = 3.0) -> Dataset:
    """Binary labels = [hidden depth-5 program > 0], 5% flipped; weight 1
    for the positive class and 3 for the negative class."""
    rng = np.random.default_rng(seed)
    # drawn in float32 (in place) so that wide tables need no float64 copy
    X = rng.random((n_feat, n_rows), dtype=np.float32)
    X *= np.float32(2.0)
    X -= np.float32(1.0)
    hid = _hidden_program(rng, depth, n_feat)
    h = _compose(hid, X)
    lab = (h > 0).astype(np.float32)
    fl = rng.random(n_rows) < flip
    lab[fl] = 1.0 - lab[fl]
    w = np.where(lab > 0.5, w_pos, w_neg).astype(np.float32)
    return Dataset(X, lab, w, f"binary_n{n_rows}_f{n_feat}", pack([hid]))


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    data: Dataset
    nodes: np.ndarray
    offsets: np.ndarray
    metric: str
    tourn_size: int
    funcs: Tuple[str, ...]


def workload(name: str, n_rows: Optional[int] = None, n_progs: Optional[int] = None) -> Workload:
    """The five evaluation workloads (data seed 1234+i, population seed 99+i).

    pagie_small : N=4096, P=512, RHH depth 2-6, {add,sub,mul,div}, MSE, k=20
    pagie_large : N=1M or 16M, P=4096, depth 2-10, 12-op set, RMSE, k=20
    tabular     : N=10M x 28, P=2048, depth 2-8, 12-op set, RMSE
    binary      : N=4M x 50, P=1024, weighted log-loss, k=10
    const_tune  : Pagie N=1M, P=2048, depth 4-10, <=16 constants, MSE
    wide        : Epsilon-shaped N=500K x 2000, P=1024, depth 2-8, log-loss, k=10
    """
    if name == "pagie_small":
        n = n_rows or 4096
        d = pagie_data(n, 1234)
        nodes, off = ramped_half_and_half(n_progs or 512, 2, 6, BASIC_SET, 2, 99)
        return Workload(name, d, nodes, off, "mse", 20, BASIC_SET)
    if name == "pagie_large":
        n = n_rows or (1 << 24)
        d = pagie_data(n, 1235)
        nodes, off = ramped_half_and_half(n_progs or 4096, 2, 10, FULL_SET, 2, 100)
        return Workload(name, d, nodes, off, "rmse", 20, FULL_SET)
    if name == "tabular":
        n = n_rows or 10_000_000
        d = tabular_data(n, 1236)
        nodes, off = ramped_half_and_half(n_progs or 2048, 2, 8, FULL_SET, 28, 101)
        return Workload(name, d, nodes, off, "rmse", 20, FULL_SET)
    if name == "binary":
        n = n_rows or (1 << 22)
        d = classification_data(n, 1237)
        nodes, off = ramped_half_and_half(n_progs or 1024, 2, 8, FULL_SET, 50, 102)
        return Workload(name, d, nodes, off, "logloss", 10, FULL_SET)
    if name == "const_tune":
        n = n_rows or (1 << 20)
        d = pagie_data(n, 1238)
        nodes, off = ramped_half_and_half(n_progs or 2048, 4, 10, FULL_SET, 2, 103,
                                          max_consts=16)
        return Workload(name, d, nodes, off, "mse", 20, FULL_SET)
    if name == "wide":
        n = n_rows or 500_000
        d = classification_data(n, 1239, n_feat=2000, depth=5)
        nodes, off = ramped_half_and_half(n_progs or 1024, 2, 8, FULL_SET, 2000, 104)
        return Workload(name, d, nodes, off, "logloss", 10, FULL_SET)
    raise KeyError(name)
