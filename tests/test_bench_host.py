"""Host logic of bench.py (CPU): the kernel-source hash that keys the
recorded DRAM traffic ignores comments and blank lines but not code, and the
recorded figure is read only while that hash matches."""
from __future__ import annotations

import bench


def test_code_only_drops_comments_and_blank_lines():
    src = """// header comment
#include "x.h"   // trailing

/* block
   comment */ int a = 1;
int b = 2; /* inline */ int c = 3;

"""
    out = bench._code_only(src)
    assert out.splitlines() == ['#include "x.h"', " int a = 1;", "int b = 2;  int c = 3;"]


def test_hash_follows_code_not_comments(monkeypatch, tmp_path):
    files = {k: "" for k in bench.KERNEL_SOURCES}
    files["gp_interp.cuh"] = "int f() { return 1; }  // one\n"
    csrc = tmp_path / "paper_2110_11226_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for k, v in files.items():
        (csrc / k).write_text(v)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_hash()
    (csrc / "gp_interp.cuh").write_text("// a new comment\n\nint f() { return 1; }  // two\n")
    assert bench.kernel_hash() == h0
    (csrc / "gp_interp.cuh").write_text("int f() { return 2; }\n")
    assert bench.kernel_hash() != h0


def test_recorded_traffic_is_keyed_by_the_hash(monkeypatch, tmp_path):
    csrc = tmp_path / "paper_2110_11226_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for k in bench.KERNEL_SOURCES:
        (csrc / k).write_text("int x;\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_hash()
    prof = tmp_path / "profiles" / "eval_kernel_pagie1_traffic.md"
    prof.write_text(f"- workload: pagie_large\n- launch_shape: 8/32/8\n"
                    f"- kernel_sources_sha256_16: {h}\n- dram_bytes_per_row: 13.5\n")
    assert bench.recorded_traffic("pagie_large", "8/32/8") == 13.5
    assert bench.recorded_traffic("tabular", "8/32/8") is None
    # another launch shape reads the inputs another number of times
    assert bench.recorded_traffic("pagie_large", "4/0/0") is None
    # several launch shapes, each figure after its own launch_shape line
    prof.write_text(f"- workload: pagie_large\n- kernel_sources_sha256_16: {h}\n"
                    f"- launch_shape: 4/0/0\n- dram_bytes_per_row: 12.5\n"
                    f"- launch_shape: 8/32/8\n- dram_bytes_per_row: 12.75\n")
    assert bench.recorded_traffic("pagie_large", "4/0/0") == 12.5
    assert bench.recorded_traffic("pagie_large", "8/32/8") == 12.75
    assert bench.recorded_traffic("pagie_large", "8/0/0") is None
    (csrc / "gp_compile.cu").write_text("int y;\n")
    assert bench.recorded_traffic("pagie_large", "4/0/0") is None


def test_traffic_launch_shape_key():
    import types
    split = types.SimpleNamespace(rows_per_thread=8, long_edge=32, long_rows_per_thread=8)
    plain = types.SimpleNamespace(rows_per_thread=4, long_edge=-1, long_rows_per_thread=8)
    assert bench.traffic_opts_key(split) == "8/32/8"
    assert bench.traffic_opts_key(plain) == "4/0/0"


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the oracle on the host cores) prints one
    JSON line with the keys the benchmark contract asks of that arm."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--workload", "pagie_small", "--n-rows", "4096", "--steps", "1",
                        "--warmup", "0", "--cpu-seconds", "1"],
                       capture_output=True, text=True, cwd=root, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    for k in ("metric", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "dtype", "config"):
        assert k in d, k
    assert d["config"]["workload"] == "pagie_small"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_clock_sampler_reads_clocks_and_throttle_reasons(monkeypatch, tmp_path):
    """The clocks record of the JSON line: median SM clock under load, the
    maximum clock, and the throttle reasons seen active, from nvidia-smi's
    CSV samples (here a stand-in script on PATH); no nvidia-smi at all gives
    an explicit "unsampled" record."""
    import os
    import time
    fake = tmp_path / "nvidia-smi"
    rows = ["0, 1900, 2070, 800.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1965, 2070, 900.1, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2010, 2070, 950.5, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbled line"]
    fake.write_text("#!/bin/sh\n" + "".join(f"echo '{r}'\n" for r in rows) + "sleep 5\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    with bench.ClockSampler(0) as c:
        for _ in range(100):
            time.sleep(0.02)
            if os.path.getsize(c.path) >= sum(len(r) + 1 for r in rows):
                break
    s = c.summary()
    assert s == {"sm_mhz": 1965.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    monkeypatch.setenv("PATH", str(tmp_path / "empty"))
    with bench.ClockSampler(0) as c:
        pass
    assert c.summary()["reasons"] == ["unsampled"]


def test_folded_op_counts_follow_the_pre_pass_folding():
    """Constant-only subtrees fold to one constant: their function nodes
    leave the count, and the folded-away nodes are counted."""
    import bench
    from helpers import pack, parse_prefix
    progs = ["sin add 0.5 0.25",            # all constant: 3 nodes folded, no function left
             "mul x0 exp 0.5",               # exp(0.5) folds: 1 node folded, mul left
             "add sqrt x0 div x1 0.5",       # nothing constant-only above a terminal
             "sub log mul 2 3 x0"]           # log(mul(2,3)) folds: 3 nodes folded
    nodes, off = pack([parse_prefix(p) for p in progs])
    n_fn, sfu, folded = bench.folded_op_counts(nodes, off)
    assert folded == 3 + 1 + 0 + 3
    assert n_fn == 0 + 1 + 3 + 1
    assert sfu.get("sin", 0) == 0 and sfu.get("ex2", 0) == 0 and sfu.get("lg2", 0) == 0
    assert sfu["rsqrt"] == 1 and sfu["rcp"] == 1


def test_workloads_run_at_their_own_size_by_default(monkeypatch):
    """Without --n-rows each workload keeps the row count it is defined
    with (16,777,216 only for pagie_large); --n-rows overrides it."""
    import sys
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "pagie_small"])
    args = bench.parse()
    assert args.n_rows == 0
    assert bench.make_workload(args, 0).data.n_rows == 4096
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "pagie_small", "--n-rows", "1000"])
    assert bench.make_workload(bench.parse(), 0).data.n_rows == 1000
