"""Resident blocks of the evaluator's common-class instances (CPU, from
ptxas's resource report): the design rests on 8 rows per lane fitting 4
blocks of 8 warps per SM (64 registers, a 6-slot stack) and 4 rows per lane
fitting 5.  A change that costs a block shows up here before any GPU run.

Per SM on the GB300: 65,536 registers, allocated per warp in units of 256
(8 per thread), and 228 KB of shared memory, of which each block also
reserves 1 KB."""
from __future__ import annotations

import os
import re
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.join(ROOT, "paper_2110_11226_gb300"))
import build  # noqa: E402

REGS_PER_SM = 65536
SMEM_PER_SM = 228 * 1024
SMEM_RESERVED_PER_BLOCK = 1024
CODE_STRIDE = 256  # instruction words per program (gp_internal.cuh)


def _resources(src, tmp_path):
    """{mangled kernel name: (registers, static shared bytes, spill loads)}"""
    nvcc = build._nvcc()
    if shutil.which(nvcc) is None and not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    r = subprocess.run([nvcc] + build.NVCC_FLAGS + ["-Xptxas", "-v", "-c",
                        os.path.join(build.CSRC, src), "-o", str(tmp_path / "x.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out, cur, spills = {}, None, {}
    for line in r.stderr.splitlines():
        m = re.search(r"Compiling entry function '(\w+)'", line)
        if m:
            cur = m.group(1)
            continue
        m = re.search(r"(\d+) bytes spill loads", line)
        if m and cur:
            spills[cur] = int(m.group(1))
        m = re.search(r"Used (\d+) registers.*?(\d+) bytes smem", line)
        if m and cur:
            out[cur] = (int(m.group(1)), int(m.group(2)), spills.get(cur, 0))
    return out


def _blocks(regs, static_smem, rpt, nslot, warps=8):
    dyn = (CODE_STRIDE + 2) * 8 + warps * nslot * (rpt // 4) * 32 * 16
    per_warp_regs = ((regs + 7) // 8) * 8 * 32
    by_regs = REGS_PER_SM // (per_warp_regs * warps)
    by_smem = SMEM_PER_SM // (dyn + static_smem + SMEM_RESERVED_PER_BLOCK)
    return min(by_regs, by_smem)


def test_common_class_fits_four_blocks_at_eight_rows(tmp_path):
    res = _resources("gp_eval_r8_f2.cu", tmp_path)
    # eval_kernel<RPT=8, NSLOT=6, FMODE=2, EPI=loss, EXT=false>
    name = next(k for k in res if "eval_kernelILi8ELi6ELi2ELi0ELb0E" in k)
    regs, smem, spill = res[name]
    assert regs <= 64, res[name]
    assert spill <= 64, res[name]  # a few words outside the word loop
    assert _blocks(regs, smem, 8, 6) >= 4, res[name]


def test_common_class_fits_five_blocks_at_four_rows(tmp_path):
    res = _resources("gp_eval_r4_f2.cu", tmp_path)
    name = next(k for k in res if "eval_kernelILi4ELi6ELi2ELi0ELb0E" in k)
    regs, smem, spill = res[name]
    assert spill == 0, res[name]
    assert _blocks(regs, smem, 4, 6) >= 5, res[name]
