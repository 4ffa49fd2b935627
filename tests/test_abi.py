"""The C ABI library: it loads, exports every entry point of include/gp.h,
agrees with the oracle and the input generator on the node format, and its
host-side validation agrees with the oracle (CPU only, no compute calls on a
GPU)."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2110_11226_gb300 import build as gpbuild
from paper_2110_11226_gb300 import synth
from helpers import parse_prefix, pack

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gp.h")


def _declared():
    with open(HEADER) as f:
        txt = f.read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gp_[a-z0-9_]+)\s*\(", txt)))


def _enum(name_prefix):
    with open(HEADER) as f:
        txt = f.read()
    return {m.group(1): int(m.group(2)) for m in re.finditer(rf"\b({name_prefix}[A-Z_0-9]+)\s*=\s*(-?\d+)", txt)}


def test_library_exports_every_declared_symbol():
    path = gpbuild.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_opcodes_agree_between_header_oracle_and_generator():
    ops = _enum("GP_")
    for name, code in synth.OP.items():
        assert ops["GP_" + name.upper()] == code, name
        assert oracle.OPS[name] == code
        assert oracle.op_name(code) == name
        assert oracle.op_arity(code) == synth.ARITY[code]
    assert ops["GP_NUM_OPS"] == len(synth.OP)
    assert ops["GP_MAE"] == 0 and ops["GP_MSE"] == 1 and ops["GP_RMSE"] == 2 and ops["GP_LOGLOSS"] == 3
    for k, v in oracle.METRICS.items():
        assert ops["GP_" + k.upper()] == v
    # gp_node is 8 bytes: int16 op, int16 feat, float c
    assert synth.NODE_DTYPE.itemsize == 8 and oracle.NODE_DTYPE == synth.NODE_DTYPE
    st = _enum("GP_PROG_")
    assert st["GP_PROG_OK"] == oracle.OK and st["GP_PROG_TOO_DEEP"] == oracle.TOO_DEEP
    assert st["GP_PROG_UNDERFLOW"] == oracle.UNDERFLOW and st["GP_PROG_LEFTOVER"] == oracle.LEFTOVER


def test_host_validation_agrees_with_oracle():
    from paper_2110_11226_gb300 import gp
    rng = np.random.default_rng(5)
    progs = []
    n_feat = 3
    good = synth.unpack(*synth.random_programs(200, 9, synth.FULL_SET + ("tan",), n_feat, seed=4))
    for p in good:
        progs.append(p)
        q = list(p)
        kind = rng.integers(6)
        if kind == 0 and len(q) > 1:
            q = q[:-1]                         # drop a terminal: underflow
        elif kind == 1:
            q = q + [(synth.OP["var"], 0, 0.0)]  # leftover value
        elif kind == 2:
            q[rng.integers(len(q))] = (77, 0, 0.0)  # unknown op
        elif kind == 3:
            q = [(synth.OP["var"], n_feat, 0.0)]    # feature out of range
        elif kind == 4:
            d = 21                                  # left spine deeper than the stack
            q = [(synth.OP["add"], 0, 0.0)] * d + [(synth.OP["var"], 0, 0.0)] + [(synth.OP["const"], 0, 1.0)] * d
        progs.append(q)
    progs.append([])
    nodes, off = pack(progs)
    rc, st, hw = gp.gp_validate_host(nodes, off, n_feat)
    assert rc == -2  # GP_ERR_PROGRAM
    for i, p in enumerate(progs):
        ost, ohw = oracle.validate(nodes[off[i]:off[i + 1]], n_feat)
        assert st[i] == ost, (i, st[i], ost)
        if ost == oracle.OK:
            assert hw[i] == ohw
    rc2, st2, _ = gp.gp_validate_host(*pack(good), n_feat)
    assert rc2 == 0 and np.all(st2 == 0)


def test_binding_signatures_match_the_header():
    """Every prototype in gp.h has a binding entry with the same number of
    arguments and the same return type, and the binding declares nothing the
    header lacks."""
    import ctypes as C
    from paper_2110_11226_gb300 import gp
    with open(HEADER) as f:
        txt = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
    protos = re.findall(r"\b(int|size_t|void|const char \*)\s*(gp_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;",
                        txt, flags=re.S)
    assert len(protos) >= 20
    ret = {"int": C.c_int, "size_t": C.c_size_t, "void": None, "const char *": C.c_char_p}
    for r, name, args in protos:
        args = " ".join(args.split())
        n_args = 0 if args in ("", "void") else args.count(",") + 1
        fn = getattr(gp._lib, name)
        assert fn.restype is ret[r], name
        assert len(fn.argtypes) == n_args, (name, len(fn.argtypes), n_args)
    bound = {n for n in dir(gp) if n.startswith("gp_")}
    assert bound <= {n for _, n, _ in protos}, bound - {n for _, n, _ in protos}


C_CLIENT = r"""
#include <stdio.h>
#include "gp.h"
int main(void) {
    gp_node prog[3] = {{GP_ADD, 0, 0.0f}, {GP_VAR, 0, 0.0f}, {GP_CONST, 0, 1.5f}};
    int32_t off[2] = {0, 3};
    int32_t st[1] = {-1}, hw[1] = {-1};
    int rc = gp_validate_host(prog, off, 1, 2, st, hw);
    printf("%s\n", gp_version());
    return (rc == GP_OK && st[0] == GP_PROG_OK && hw[0] == 2 && sizeof(gp_node) == 8) ? 0 : 1;
}
"""


def test_header_is_plain_c_and_a_c_program_links(tmp_path):
    """gp.h compiles as pedantic C99 with no CUDA or torch headers, and a C
    program links libgp and calls an entry point that needs no GPU."""
    import subprocess
    lib = gpbuild.build()
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(lib)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                    "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lgp",
                    f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("libgp"), (r.returncode, r.stdout, r.stderr)


def test_argument_errors_return_before_any_device_call():
    """Bad arguments come back as GP_ERR_ARG before the library touches CUDA;
    arguments that pass every check reach the device lookup, which on a
    machine without a GPU fails with GP_ERR_CUDA (no CPU fallback).  Runs
    only where no GPU is visible, so the placeholder pointers can never
    reach a kernel."""
    import ctypes as C
    import torch
    if torch.cuda.is_available():
        pytest.skip("placeholder pointers are only safe without a GPU")
    from paper_2110_11226_gb300 import gp
    lib = gp._lib
    ARG, CUDA = -1, -4
    buf = (C.c_uint8 * 4096)()
    p = C.cast(buf, C.c_void_p)
    ev = lambda **k: lib.gp_evaluate(k.get("progs", p), k.get("off", p), k.get("P", 4), p,
                                     k.get("N", 100), k.get("F", 2), k.get("y", p), None,
                                     k.get("metric", 1), k.get("out", p), None)
    for bad in (dict(progs=None), dict(off=None), dict(P=0), dict(N=0), dict(F=0), dict(F=32768),
                dict(N=(1 << 40) + 1), dict(y=None), dict(out=None), dict(metric=6),
                dict(metric=-1)):
        assert ev(**bad) == ARG, bad
    assert ev() == CUDA
    plain = lambda m: lib.gp_evaluate_plain(p, p, 4, p, 100, 2, p, None, m, p, None)
    assert plain(4) == ARG and plain(5) == ARG and plain(1) == CUDA
    assert lib.gp_const_grad(p, p, 4, p, 100, 2, p, None, 4, p, p, None) == ARG
    assert lib.gp_predict(p, p, 4, p, 100, 2, None, None) == ARG
    assert lib.gp_predict_ex(p, p, 4, p, 100, 2, None, None, None) == ARG
    opt = gp.make_opts(rows_per_thread=16)
    assert lib.gp_predict_ex(p, p, 4, p, 100, 2, C.byref(opt), p, None) == ARG
    assert lib.gp_predict_ex(p, p, 4, p, 100, 2, None, p, None) == CUDA
    tour = lambda **k: lib.gp_tournament_ex(k.get("fit", p), None, k.get("P", 4), k.get("T", 4),
                                            k.get("k", 2), 0.0, 0, 1, 0, k.get("out", p), None)
    for bad in (dict(fit=None), dict(out=None), dict(P=0), dict(T=-1), dict(k=0)):
        assert tour(**bad) == ARG, bad
    adam = lambda step=1, b1=0.9, b2=0.999, eps=1e-8: lib.gp_adam_step(
        p, p, 4, p, p, p, step, 1e-2, b1, b2, eps, None)
    assert adam(step=0) == ARG and adam(b1=1.0) == ARG and adam(b2=-0.1) == ARG
    assert adam(eps=0.0) == ARG
    good = dict(p_crossover=0.7, p_subtree=0.1, p_hoist=0.05, p_point=0.1, p_replace=0.1,
                subtree_depth=4)
    mut = lambda params, n_out=4: lib.gp_mutate(p, p, 4, 2, p, n_out, C.byref(params), 1, 0,
                                                p, p, None, None, 0, None)
    assert mut(gp.make_mut_params(**good)) == CUDA
    assert mut(gp.make_mut_params(**good), n_out=0) == ARG
    for bad in (dict(p_crossover=0.9, p_subtree=0.2), dict(subtree_depth=7), dict(functions=()),
                dict(p_replace=1.5), dict(p_hoist=-0.1)):
        assert mut(gp.make_mut_params(**{**good, **bad})) == ARG, bad
    q = gp.make_mut_params(**good)
    q.reserved[2] = 1
    assert mut(q) == ARG
    assert lib.gp_workspace_size(0, 100, 2, None) == 0
    assert lib.gp_mutate_workspace_size(0) == 0 and lib.gp_mutate_workspace_size((1 << 22) + 1) == 0


def test_build_targets_sm_103a_only_and_covers_every_source():
    """One -gencode for sm_103a with line info, no host-specific flags, and
    an object in the library for every .cu file of csrc/."""
    flags = gpbuild.NVCC_FLAGS
    gencodes = [flags[i + 1] for i, f in enumerate(flags) if f == "-gencode"]
    assert gencodes == ["arch=compute_103a,code=sm_103a"]
    assert "-lineinfo" in flags and not any("march" in f or "arch=sm_" in f for f in flags)
    gpbuild.build()
    for s in gpbuild.sources():
        o = os.path.join(gpbuild.BUILD, os.path.basename(s)[:-3] + ".o")
        assert os.path.exists(o) and os.path.getmtime(o) <= os.path.getmtime(gpbuild.LIB), s
    assert len(gpbuild.sources()) >= 15
