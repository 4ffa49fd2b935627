"""Benchmark: one GP generation's hot path on the GPU (arXiv 2110.11226).

A step = batched fitness evaluation of the whole population over every row
(device pre-pass + persistent evaluator with the fused loss + FP64 reduction)
followed by tournament selection on the device.  Default workload: Pagie-1,
N = 16,777,216 rows x 2 features, P = 4096 programs (ramped half-and-half,
depth 2-10, 12-op function set), RMSE, tournament size 20.

Prints one JSON line.  `value` = program-row evaluations per second with the
inputs resident in HBM; `e2e` = the same through gp_evaluate_host (host
buffers, all copies inside the timed region); `plain` = the one-launch-per-
program evaluator on the same GPU; `roofline` = the evaluator kernel against
the ALU roofline (node operations over FP32-pipe / SFU peaks, or feature
bytes over HBM bandwidth); `cpu_baseline` = the FP64 C oracle on the host
cores, on a bounded sample.

Multi-GPU (torchrun): the population is sharded by programs -- every rank
evaluates its own P programs of a global population of world*P (seed offset
by rank) on the same data, the fitness shards are all-gathered (selection
needs all of them), and every rank runs the same world*P tournaments; the
time is the max over ranks (weak scaling: P per GPU is fixed).

--impl reference: times the oracle instead (the CPU reference arm).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "program-row evals/s (GPops/s) and % roofline, batched vs plain eval, same GB300"
UNIT = "program-row evals/s"
# one special-function-unit operation per node of these ops, on this MUFU
# function (div and inv: reciprocal; sqrt: reciprocal square root; log: lg2;
# exp: ex2; sin, cos, tan: sin)
SFU_OF_OP = {5: "rcp", 14: "rcp", 6: "rsqrt", 7: "lg2", 8: "ex2", 9: "sin", 10: "sin", 11: "sin"}
LOSS_FP32 = {"mae": 3, "mse": 3, "rmse": 3, "logloss": 6}
LOSS_SFU = {"mae": {}, "mse": {}, "rmse": {}, "logloss": {"ex2": 1, "lg2": 1}}
KERNEL_SOURCES = ("gp_interp.cuh", "gp_fast.cuh", "gp_math.cuh", "gp_internal.cuh", "gp_compile.cu")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="pagie_large")
    ap.add_argument("--n-rows", type=int, default=0,
                    help="rows (0: the workload's own size; 16,777,216 for pagie_large)")
    ap.add_argument("--n-progs", type=int, default=0)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-generation", action="store_true",
                    help="skip the whole-generation (evaluate, select, mutate) timing")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip gp_autotune and run the library's default tunables")
    ap.add_argument("--rows-per-thread", type=int, default=0,
                    help="evaluator rows per thread (4, 8 or 16; 0: the library's default)")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the accumulator-error block (oracle on 16 sampled programs)")
    ap.add_argument("--chunk-rows", type=int, default=0,
                    help="rows per work item (0: the library's choice)")
    ap.add_argument("--long-edge", type=int, default=0,
                    help="length-bucket edge in compiled words (0: the library's choice)")
    ap.add_argument("--long-rows-per-thread", type=int, default=0)
    ap.add_argument("--blocks-per-sm", type=int, default=0,
                    help="resident evaluator blocks per SM (0: as many as fit)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the step eagerly instead of replaying its CUDA graph")
    ap.add_argument("--const-tune", action="store_true",
                    help="time constant tuning (fitness and gradient, then Adam) on the "
                         "const_tune workload instead (one JSON line of its own)")
    ap.add_argument("--spearman", action="store_true",
                    help="time the Spearman rank fitness on the workload instead (one JSON "
                         "line of its own, not the headline)")
    return ap.parse_args()


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_workload(args, rank):
    from paper_2110_11226_gb300 import synth
    wl = synth.workload(args.workload, n_rows=args.n_rows or None, n_progs=args.n_progs or None)
    if rank:
        # program shard of rank r: its own P programs, same data
        nodes, off = synth.ramped_half_and_half(len(wl.offsets) - 1, *_depths(args.workload),
                                                wl.funcs, wl.data.n_feat, 1000 + rank)
        wl.nodes, wl.offsets = nodes, off
    return wl


def _depths(name):
    return {"pagie_small": (2, 6), "pagie_large": (2, 10), "tabular": (2, 8),
            "binary": (2, 8), "const_tune": (4, 10)}[name]


def op_counts(nodes):
    """(function nodes, {mufu function: nodes}, all nodes) of a population."""
    op = nodes["op"].astype(np.int64)
    sfu = {}
    for code, fn in SFU_OF_OP.items():
        sfu[fn] = sfu.get(fn, 0) + int((op == code).sum())
    return int((op >= 2).sum()), sfu, int(len(op))


def folded_op_counts(nodes, offsets):
    """The pre-pass folds every maximal constant-only subtree (no variable
    below it) into one constant.  Returns (function nodes left, {mufu
    function: nodes left}, nodes folded away) -- the work the evaluator
    actually does."""
    from paper_2110_11226_gb300 import synth
    op = nodes["op"].astype(np.int64)
    var, const = synth.OP["var"], synth.OP["const"]
    n_fn = 0
    sfu = {}
    folded = 0
    for p in range(len(offsets) - 1):
        a, b = int(offsets[p]), int(offsets[p + 1])
        ops = op[a:b]
        kon = np.zeros(b - a, bool)
        size = np.ones(b - a, np.int64)
        st = []
        for j in range(b - a - 1, -1, -1):
            ar = synth.ARITY.get(int(ops[j]), -1)
            if ar == 0:
                kon[j] = ops[j] == const
            elif ar == 1:
                s1, k1 = st.pop()
                kon[j], size[j] = k1, 1 + s1
            elif ar == 2:
                s1, k1 = st.pop()
                s2, k2 = st.pop()
                kon[j], size[j] = k1 and k2, 1 + s1 + s2
            else:
                break
            st.append((size[j], kon[j]))
        inside = np.zeros(b - a, bool)
        j = 0
        while j < b - a:
            if kon[j] and ops[j] not in (var, const):  # a folded subtree: its root becomes a constant
                inside[j:j + size[j]] = True
                folded += int(size[j]) - 1
                j += int(size[j])
            else:
                j += 1
        live = ops[~inside]
        n_fn += int((live >= 2).sum())
        for code, fn in SFU_OF_OP.items():
            sfu[fn] = sfu.get(fn, 0) + int((live == code).sum())
    return n_fn, sfu, folded


def _code_only(text):
    """C++ source without its comments (the string literals of these files
    hold no comment markers), so that editing a comment keeps the hash."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (line.split("//", 1)[0].rstrip() for line in text.splitlines())
    return "\n".join(line for line in lines if line)


def kernel_hash():
    """Hash of the evaluator's sources, comments removed: the recorded DRAM
    traffic holds only for the code it was measured on."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2110_11226_gb300", "csrc", f)) as fh:
            text = fh.read()
        h.update(_code_only(text).encode())
    return h.hexdigest()[:16]


DATA_DESC = {
    "pagie_small": "synthetic: seeded Pagie-1 rows, ramped half-and-half population",
    "pagie_large": "synthetic: seeded Pagie-1 rows, ramped half-and-half population",
    "const_tune": "synthetic: seeded Pagie-1 rows, ramped half-and-half population",
    "tabular": "synthetic: seeded Higgs-shaped 28-column table, hidden-program target",
    "binary": "synthetic: seeded 50-column table, hidden-program labels, 5% flipped",
    "wide": "synthetic: seeded Epsilon-shaped 2000-column table, hidden-program labels, 5% flipped",
}


def traffic_opts_key(used):
    """The launch shape a recorded traffic figure holds for: rows per
    thread, length-bucket edge (0: no split) and the long bucket's rows per
    thread (each evaluator launch reads the inputs once)."""
    edge = used.long_edge if used.long_edge > 0 else 0
    return f"{used.rows_per_thread}/{edge}/{used.long_rows_per_thread if edge else 0}"


def recorded_traffic(workload, opts_key):
    """DRAM bytes per row of the evaluator from the committed ncu summary, if
    it was taken on the current kernel sources and launch shape (else
    None)."""
    path = os.path.join(ROOT, "profiles", "eval_kernel_pagie1_traffic.md")
    if not os.path.exists(path):
        return None
    vals, per_shape, shape = {}, {}, None
    with open(path) as fh:
        for line in fh:
            if ":" in line and line.startswith("- "):
                k, v = line[2:].split(":", 1)
                k, v = k.strip(), v.strip().strip("`")
                vals[k] = v
                # each launch shape's figure follows its own launch_shape line
                if k == "launch_shape":
                    shape = v
                elif k == "dram_bytes_per_row" and shape is not None:
                    per_shape[shape] = v
    if vals.get("kernel_sources_sha256_16") != kernel_hash() or vals.get("workload") != workload \
            or opts_key not in per_shape:
        return None
    try:
        return float(per_shape[opts_key])
    except ValueError:
        return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            with open(self.path, "w") as out:
                self.proc = subprocess.Popen(
                    ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                     "--format=csv,noheader,nounits", "-lms", "200"],
                    stdout=out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            with open(self.path) as fh:
                lines = fh.readlines()
            for line in lines:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    rows.append((float(f[1]), float(f[2]), f[5:9]))
                except ValueError:
                    continue
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        load = [r[0] for r in rows]
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(wl, seconds, n_threads=0):
    """The oracle as it stands, on a bounded sample of the workload."""
    import oracle
    d = wl.data
    P = len(wl.offsets) - 1
    # calibrate on a small sample, then size the measured one to ~`seconds`
    n0 = min(d.n_rows, 1 << 14)
    p0 = min(P, 64)
    t = time.perf_counter()
    oracle.fitness(wl.nodes, wl.offsets[:p0 + 1], d.X, d.y, d.w, wl.metric, n_eval=n0,
                   n_threads=n_threads)
    dt = max(time.perf_counter() - t, 1e-4)
    rate = p0 * n0 / dt
    n_s = int(min(d.n_rows, max(n0, seconds * rate / p0)))
    t = time.perf_counter()
    oracle.fitness(wl.nodes, wl.offsets[:p0 + 1], d.X, d.y, d.w, wl.metric, n_eval=n_s,
                   n_threads=n_threads)
    dt = time.perf_counter() - t
    return {"value": p0 * n_s / dt, "unit": UNIT, "cores": oracle.max_threads() if n_threads <= 0 else n_threads,
            "kind": "oracle",
            "sample": f"first {p0} programs x first {n_s} rows of {wl.name}, FP64 C oracle, OpenMP over programs",
            "seconds": round(dt, 2)}


def precision_block(wl, pn, po, dX, dy, dw, opts, k=16):
    """Error of the fitness against the FP64 oracle over every row, for each
    cross-chunk accumulator (FP64, Kahan FP32), on k sampled programs whose
    oracle fitness is finite."""
    import oracle
    from paper_2110_11226_gb300 import gp
    d = wl.data
    P = len(wl.offsets) - 1
    res = {}
    fits = {}
    for acc in ("fp64", "kahan32"):
        o = gp.make_opts(rows_per_thread=opts.rows_per_thread, chunk_rows=opts.chunk_rows,
                         blocks_per_sm=opts.blocks_per_sm, accum=acc)
        fits[acc] = gp.gp_evaluate_ex(pn, po, dX, dy, dw, metric=wl.metric, opts=o).cpu().numpy()
    idx = np.sort(np.random.default_rng(17).choice(P, size=min(k, P), replace=False))
    progs = [wl.nodes[wl.offsets[i]:wl.offsets[i + 1]] for i in idx]
    sn = np.concatenate(progs)
    so = np.zeros(len(idx) + 1, np.int32)
    so[1:] = np.cumsum([len(x) for x in progs])
    f64, _ = oracle.fitness(sn, so, d.X, d.y, d.w, wl.metric)
    fin = np.isfinite(f64) & np.isfinite(fits["fp64"][idx])
    for acc, f in fits.items():
        with np.errstate(all="ignore"):
            rel = np.abs(f[idx][fin] - f64[fin]) / np.maximum(np.abs(f64[fin]), 1e-300)
        res[acc] = {"max_rel": float(rel.max()) if rel.size else None,
                    "median_rel": float(np.median(rel)) if rel.size else None}
    with np.errstate(all="ignore"):
        both = np.isfinite(fits["fp64"]) & np.isfinite(fits["kahan32"])
        diff = np.abs(fits["fp64"][both] - fits["kahan32"][both]) / \
            np.maximum(np.abs(fits["fp64"][both]), 1e-300)
    res["fp64_vs_kahan32_max_rel"] = float(diff.max()) if diff.size else None
    res["programs_compared"] = int(fin.sum())
    res["reference"] = (f"FP64 C oracle over all {d.n_rows} rows of {len(idx)} sampled programs "
                        f"(finite ones compared); GPU rows in FP32, per-lane Kahan FP32, chunk "
                        f"sums in FP64 or Kahan FP32")
    return res


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    wl = make_workload(args, 0)
    import oracle
    P = len(wl.offsets) - 1
    vals = []
    for s in range(args.warmup + args.steps):
        r = cpu_baseline(wl, max(1.0, min(args.cpu_seconds, 20.0) / max(args.steps, 1)))
        if s >= args.warmup:
            vals.append(r["value"])
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * P * wl.data.n_rows / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": DATA_DESC.get(wl.name, "synthetic, seeded"),
            "config": {"workload": wl.name, "n_rows": wl.data.n_rows,
                                            "n_progs": P, "n_feat": wl.data.n_feat, "metric": wl.metric},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_spearman(args):
    """Spearman rank fitness (batched predictions, radix sort, ranks) of the
    workload's population, timed with CUDA events around gp_evaluate."""
    import torch
    from paper_2110_11226_gb300 import gp
    wl = make_workload(args, 0)
    d = wl.data
    P, N = len(wl.offsets) - 1, d.n_rows
    pn = gp.nodes_to_device(wl.nodes)
    po = torch.from_numpy(wl.offsets).cuda()
    dX, dy = torch.from_numpy(d.X).cuda(), torch.from_numpy(d.y).cuda()
    dw = None if d.w is None else torch.from_numpy(d.w).cuda()
    out = torch.empty(P, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        gp.gp_evaluate(pn, po, dX, dy, dw, metric="spearman", out=out)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        gp.gp_evaluate(pn, po, dX, dy, dw, metric="spearman", out=out)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.steps
    print(json.dumps({"metric": "Spearman fitness program-rows/s", "value": P * N / (ms * 1e-3),
                      "unit": "program-row evals/s", "ms_per_step": ms, "steps": args.steps,
                      "warmup": args.warmup, "data": DATA_DESC.get(wl.name, "synthetic"),
                      "config": {"workload": wl.name, "n_rows": N, "n_progs": P,
                                 "n_feat": d.n_feat, "metric": "spearman"}}))


def run_const_tune(args):
    """Constant tuning on the const_tune workload (Pagie-1 1M rows x 2048
    programs with up to 16 constants, MSE): a step is 5 x (fitness and
    gradient of every program's constants in one pass, then one Adam step),
    timed with CUDA events; the fitness-only evaluation is timed beside it."""
    import torch
    from paper_2110_11226_gb300 import gp
    args.workload = "const_tune"
    wl = make_workload(args, 0)
    d = wl.data
    P, N = len(wl.offsets) - 1, d.n_rows
    pn = gp.nodes_to_device(wl.nodes)
    po = torch.from_numpy(wl.offsets).cuda()
    dX, dy = torch.from_numpy(d.X).cuda(), torch.from_numpy(d.y).cuda()
    grad = torch.empty((P, gp.MAX_CONSTS), dtype=torch.float32, device="cuda")
    fit = torch.empty(P, dtype=torch.float32, device="cuda")
    m = torch.zeros_like(grad)
    v = torch.zeros_like(grad)
    inner = 5

    def step(k):
        for i in range(inner):
            gp.gp_const_grad(pn, po, dX, dy, metric=wl.metric, out_grad=grad, out_fitness=fit)
            gp.gp_adam_step(pn, po, grad, m, v, k * inner + i + 1, lr=1e-2)

    def timed(fn, reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for k in range(reps):
            fn(k)
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    ms = timed(lambda k: step(args.warmup + k), args.steps)
    grad_ms = timed(lambda k: gp.gp_const_grad(pn, po, dX, dy, metric=wl.metric, out_grad=grad,
                                               out_fitness=fit), args.steps)
    adam_ms = timed(lambda k: gp.gp_adam_step(pn, po, grad, m, v, 1000 + k, lr=1e-2), args.steps)
    eval_ms = timed(lambda k: gp.gp_evaluate(pn, po, dX, dy, metric=wl.metric, out=fit), args.steps)
    print(json.dumps({"metric": "constant-tuning program-row gradient evals/s",
                      "value": inner * P * N / (ms * 1e-3), "unit": "program-row evals/s",
                      "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
                      "grad_ms": grad_ms, "adam_ms": adam_ms, "eval_ms": eval_ms,
                      "grad_over_eval": grad_ms / eval_ms,
                      "step": f"{inner} x (gp_const_grad + gp_adam_step), eager launches",
                      "data": DATA_DESC.get(wl.name, "synthetic"),
                      "config": {"workload": wl.name, "n_rows": N, "n_progs": P,
                                 "n_feat": d.n_feat, "metric": wl.metric}}))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.spearman:
        return run_spearman(args)
    if args.const_tune:
        return run_const_tune(args)
    import torch
    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2110_11226_gb300 import gp

    wl = make_workload(args, rank)
    d = wl.data
    P = len(wl.offsets) - 1
    N = d.n_rows
    dev = torch.device("cuda", local)
    pn = gp.nodes_to_device(wl.nodes, dev)
    po = torch.from_numpy(wl.offsets).to(dev)
    dX = torch.from_numpy(d.X).to(dev)
    dy = torch.from_numpy(d.y).to(dev)
    dw = None if d.w is None else torch.from_numpy(d.w).to(dev)
    fit = torch.empty(P, dtype=torch.float32, device=dev)
    win = torch.empty(ws * P, dtype=torch.int32, device=dev)
    from paper_2110_11226_gb300.dist import gather_fitness
    stream = torch.cuda.current_stream()
    pipes = gp.gp_probe_pipes()
    # the tunables: gp_autotune's choice for this shape (on the first 2^21
    # rows) unless asked otherwise; the defaults are timed beside it below
    tuned = None
    tune_s = None
    # the library defaults for this shape, taken before any tuning record
    # exists (blocks_per_sm 32 = as many as fit; no length split)
    dflt_used = gp.gp_resolve_opts(P, N, d.n_feat, None)
    dflt_used.blocks_per_sm = 32
    dflt_used.long_edge = -1
    dflt_used.long_blocks_per_sm = 32
    explicit = args.rows_per_thread or args.blocks_per_sm or args.long_edge or args.chunk_rows
    if not args.no_autotune and not explicit:
        t0 = time.perf_counter()
        tuned = gp.gp_autotune(pn, po, dX, dy, dw, metric=wl.metric)
        tune_s = time.perf_counter() - t0

    # the generation step: batched evaluation (pre-pass, persistent
    # evaluator, FP64 finalize) and tournament selection, captured once as a
    # CUDA graph on a preallocated workspace and replayed (or launched
    # eagerly with --no-graph); with several ranks the fitness all-gather
    # sits between the two and the step runs eagerly
    opts = tuned if tuned is not None else gp.make_opts(
        rows_per_thread=args.rows_per_thread, blocks_per_sm=args.blocks_per_sm,
        chunk_rows=args.chunk_rows, long_edge=args.long_edge,
        long_rows_per_thread=args.long_rows_per_thread)
    ws_buf = torch.empty(gp.gp_workspace_size(P, N, d.n_feat, opts), dtype=torch.uint8, device=dev)
    used = gp.gp_resolve_opts(P, N, d.n_feat, opts)

    def step_eager(seed):
        gp.gp_evaluate_ex(pn, po, dX, dy, dw, metric=wl.metric, opts=opts, out=fit, ws=ws_buf)
        gfit = gather_fitness(fit) if ws > 1 else fit
        gp.gp_tournament_ex(gfit, ws * P, wl.tourn_size, seed, out=win)

    use_graph = not args.no_graph and ws == 1
    graph = None
    if use_graph:
        gstream = torch.cuda.Stream()
        gstream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(gstream):
            step_eager(42)  # warm the path on the capture stream
        gstream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=gstream):
            step_eager(42)
        torch.cuda.synchronize()

    def step(seed):
        if graph is not None:
            graph.replay()
        else:
            step_eager(seed)

    for s in range(args.warmup):
        step(42 + s)
    torch.cuda.synchronize()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for s in range(args.steps):
            step(1000 + s)
        e1.record(stream)
        torch.cuda.synchronize()
    total_ms = e0.elapsed_time(e1)
    # the evaluator kernels alone (events around its launches, on its stream)
    gp.gp_timing_enable(True)
    for s in range(min(args.steps, 3)):
        step_eager(2000 + s)
    eval_ms, n_eval_calls = gp.gp_timing_read()
    gp.gp_timing_enable(False)
    # the library defaults on the same step (eager launches), for comparison
    untuned = None
    if tuned is not None:
        dws = torch.empty(gp.gp_workspace_size(P, N, d.n_feat, dflt_used), dtype=torch.uint8,
                          device=dev)

        def step_default(seed):
            gp.gp_evaluate_ex(pn, po, dX, dy, dw, metric=wl.metric, opts=dflt_used, out=fit, ws=dws)
            gp.gp_tournament_ex(fit, ws * P, wl.tourn_size, seed, out=win)

        step_default(5)
        torch.cuda.synchronize()
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        kd = max(1, min(args.steps, 3))
        a_.record(stream)
        for s_ in range(kd):
            step_default(3000 + s_)
        b_.record(stream)
        torch.cuda.synchronize()
        untuned = {"ms_per_step": a_.elapsed_time(b_) / kd,
                   "opts": {"rows_per_thread": dflt_used.rows_per_thread,
                            "chunk_rows": dflt_used.chunk_rows, "long_edge": None},
                   "step": "eager launches, library defaults"}
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    clocks = clk.summary()
    rows_evals = float(N) * P
    value = ws * rows_evals * args.steps / (total_ms * 1e-3)
    fin = torch.isfinite(fit).float().mean().item()

    # roofline of the evaluator kernel (per launch = one population over N
    # rows): node operations over the FP32-pipe and special-function-unit
    # rates measured in this run, or feature bytes over HBM bandwidth
    n_fn, sfu_counts, n_nodes = op_counts(wl.nodes)
    for fn, k in LOSS_SFU[wl.metric].items():
        sfu_counts[fn] = sfu_counts.get(fn, 0) + k * P
    n_sfu = sum(sfu_counts.values())
    ops_fp32 = N * (n_fn + LOSS_FP32[wl.metric] * P)
    ops_sfu = N * n_sfu
    t_sfu = sum(N * k / pipes[fn] for fn, k in sfu_counts.items())
    bytes_alg = N * 4 * (d.n_feat + 1 + (d.w is not None))
    peak_fp32 = pipes["fp32"]
    peak_sfu = ops_sfu / t_sfu if t_sfu > 0 else pipes["ex2"]  # this op mix's rate
    hbm = 6800.0
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            hbm = json.load(fh)["hbm_gbs"]
    t_kernel = eval_ms / max(n_eval_calls, 1) * 1e-3
    cands = {"fp32": ops_fp32 / peak_fp32, "sfu": t_sfu, "hbm": bytes_alg / (hbm * 1e9)}
    bound = max(cands, key=cands.get)
    if bound == "hbm":
        roof = {"bound": "hbm", "achieved": bytes_alg / t_kernel / 1e9, "peak": hbm, "unit": "GB/s"}
    else:
        ops = ops_fp32 if bound == "fp32" else ops_sfu
        pk = peak_fp32 if bound == "fp32" else peak_sfu
        roof = {"bound": "alu", "pipe": bound, "achieved": ops / t_kernel / 1e12,
                "peak": pk / 1e12, "unit": "Tlane-op/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # the same on the work left after constant folding (the folded nodes are
    # evaluated once per program, not per row)
    n_fn_e, sfu_e, n_folded = folded_op_counts(wl.nodes, wl.offsets)
    for fn, kk in LOSS_SFU[wl.metric].items():
        sfu_e[fn] = sfu_e.get(fn, 0) + kk * P
    if bound != "hbm":
        if bound == "fp32":
            ops_e = N * (n_fn_e + LOSS_FP32[wl.metric] * P)
        else:
            ops_e = N * sum(sfu_e.values())
            t_sfu_e = sum(N * kk / pipes[fn] for fn, kk in sfu_e.items())
            pk = ops_e / t_sfu_e if t_sfu_e > 0 else pk
        roof["achieved_evaluated"] = ops_e / t_kernel / 1e12
        roof["peak_evaluated"] = pk / 1e12
        roof["frac_evaluated"] = roof["achieved_evaluated"] / roof["peak_evaluated"]
    roof["folded_nodes"] = n_folded
    tpr = recorded_traffic(wl.name, traffic_opts_key(used))
    roof["traffic"] = None if tpr is None else tpr * N
    roof["algorithmic_bytes"] = bytes_alg
    roof["kernel_ms"] = t_kernel * 1e3
    roof["t_roof_ms"] = {k: v * 1e3 for k, v in cands.items()}
    roof["sfu_ops_by_function"] = {k: v * N for k, v in sfu_counts.items()}
    roof["peak_source"] = ("gp_probe_pipes in this run: FADD and MUFU ex2/rcp/rsqrt/lg2/sin chains on "
                           "all SMs at the running clock; SFU peak = this op mix's rate")
    roof["kernel_sources_sha256_16"] = kernel_hash()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": DATA_DESC.get(wl.name, "synthetic, seeded"),
            "config": {"workload": wl.name, "n_rows": N, "n_feat": d.n_feat, "n_progs": P,
                       "metric": wl.metric, "tourn_size": wl.tourn_size,
                       "mean_nodes": n_nodes / P, "function_nodes": n_fn, "sfu_nodes": n_sfu,
                       "step": "cuda graph replay" if graph is not None else "eager launches",
                       "l2": "inputs larger than L2" if N * 4 * (d.n_feat + 1) > 129e6 else "L2-resident inputs",
                       "parallelism": f"program shards x{ws} + fitness all-gather" if ws > 1 else "single GPU",
                       "opts": {"rows_per_thread": used.rows_per_thread, "chunk_rows": used.chunk_rows,
                                "blocks_per_sm": used.blocks_per_sm or "max resident",
                                "long_edge": used.long_edge if used.long_edge > 0 else None,
                                "long_rows_per_thread": used.long_rows_per_thread if used.long_edge > 0 else None,
                                "long_blocks_per_sm": (used.long_blocks_per_sm or "max resident")
                                if used.long_edge > 0 else None,
                                "classes_1_to_3_rows_per_thread": 4, "autotuned": tuned is not None,
                                "autotune_seconds": tune_s, "untuned": untuned}},
            "node_evals_per_s": value * (n_nodes / P),
            "finite_fitness_frac": fin,
            "clocks": clocks,
            # per step: compile, order, weight sum (+1 with weights), four
            # evaluator launches (program classes; +1 when the common class is
            # split by length), finalize, tournament
            "gpu_launches": (9 + (d.w is not None) + (used.long_edge > 0)) * args.steps,
            "roofline": roof,
            "pipes": pipes}

    if rank == 0 and not args.no_plain:
        gp.gp_evaluate_plain(pn, po, dX, dy, dw, metric=wl.metric, out=fit)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        gp.gp_evaluate_plain(pn, po, dX, dy, dw, metric=wl.metric, out=fit)
        b.record(stream)
        torch.cuda.synchronize()
        pms = a.elapsed_time(b)
        line["plain"] = {"value": rows_evals / (pms * 1e-3), "unit": UNIT, "ms_per_eval": pms,
                         "launches": P + 3}
        line["batched_over_plain"] = value / ws / line["plain"]["value"]

    if rank == 0 and ws == 1 and not args.no_generation:
        # a whole generation on the device (evaluate, 2 tournaments per
        # offspring, mutate into a new packed population), one CUDA graph;
        # reported beside the headline step, which is evaluation + selection
        win2 = torch.empty(2 * P, dtype=torch.int32, device=dev)
        mparams = gp.make_mut_params()
        mws = torch.empty(gp.gp_mutate_workspace_size(P), dtype=torch.uint8, device=dev)
        mout = torch.empty(P * 255, dtype=torch.int64, device=dev)
        moff = torch.empty(P + 1, dtype=torch.int32, device=dev)
        mkind = torch.empty(P, dtype=torch.int32, device=dev)

        def mutate(seed):
            gp.gp_mutate(pn, po, d.n_feat, win2, mparams, seed=seed, offset=1, out=mout,
                         out_offsets=moff, out_kind=mkind, ws=mws)

        def gen_eager(seed):
            gp.gp_evaluate_ex(pn, po, dX, dy, dw, metric=wl.metric, opts=opts, out=fit, ws=ws_buf)
            gp.gp_tournament_ex(fit, 2 * P, wl.tourn_size, seed, out=win2)
            mutate(seed + 1)

        gs2 = torch.cuda.Stream()
        gs2.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(gs2):
            gen_eager(7)
        gs2.synchronize()
        ggraph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(ggraph, stream=gs2):
            gen_eager(7)
        torch.cuda.synchronize()
        ggraph.replay()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        kg = max(1, min(args.steps, 3))
        a.record(stream)
        for _ in range(kg):
            ggraph.replay()
        b.record(stream)
        torch.cuda.synchronize()
        gms = a.elapsed_time(b) / kg
        a.record(stream)
        for s in range(5):
            mutate(30 + s)
        b.record(stream)
        torch.cuda.synchronize()
        line["full_generation"] = {
            "ms": gms, "program_rows_per_s": rows_evals / (gms * 1e-3),
            "mutate_ms": a.elapsed_time(b) / 5,
            "new_nodes": int(moff[-1].item()),
            "kinds": {k: int((mkind == v).sum().item()) for k, v in gp.MUT_KINDS.items()},
            "step": "cuda graph: evaluate, 2 tournaments per offspring, gp_mutate"}

    if rank == 0 and not args.no_e2e:
        hn = wl.nodes
        ho = wl.offsets
        hX = torch.from_numpy(d.X).pin_memory().numpy()
        hy = torch.from_numpy(d.y).pin_memory().numpy()
        hw = None if d.w is None else torch.from_numpy(d.w).pin_memory().numpy()
        hfit = torch.empty(P, dtype=torch.float32).pin_memory().numpy()
        hwin = torch.empty(P, dtype=torch.int32).pin_memory()
        fit_d = torch.empty(P, dtype=torch.float32, device=dev)

        def e2e_step(seed):
            gp.gp_evaluate_host(hn, ho, hX, hy, hw, metric=wl.metric, out=hfit)
            fit_d.copy_(torch.from_numpy(hfit), non_blocking=True)
            gp.gp_tournament_ex(fit_d, P, wl.tourn_size, seed, out=win)
            hwin.copy_(win[:P], non_blocking=True)
            torch.cuda.current_stream().synchronize()

        e2e_step(1)
        t0 = time.perf_counter()
        ksteps = max(1, min(args.steps, 3))
        for s in range(ksteps):
            e2e_step(2 + s)
        dt = time.perf_counter() - t0
        h2d = hn.nbytes + ho.nbytes + hX.nbytes + hy.nbytes + (0 if hw is None else hw.nbytes) + hfit.nbytes
        d2h = hfit.nbytes + P * 4
        line["e2e"] = {"value": rows_evals * ksteps / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                       "d2h_bytes_per_step": int(d2h), "steps": ksteps,
                       "api": "gp_evaluate_host + gp_tournament_ex (host buffers, pinned)"}

    if rank == 0 and not args.no_precision:
        line["precision"] = precision_block(wl, pn, po, dX, dy, dw, opts)

    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds)

    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
