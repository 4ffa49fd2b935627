"""The evaluator's generated and fitted sources (CPU): the inline-PTX fast
loop in gp_fast.cuh is exactly what gen_fast.py writes, and every
polynomial coefficient and constant split that gp_math.cuh pins with a
static_assert (and that the loop spells as a bit pattern) is the float32
that fit_trig.py, fit_log.py and fit_exp.py derive."""
from __future__ import annotations

import importlib.util
import os
import re
import shutil
import subprocess
import sys

import numpy as np

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2110_11226_gb300", "csrc")


def _load(name):
    spec = importlib.util.spec_from_file_location(name, os.path.join(CSRC, name + ".py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _pinned_bits():
    """{constant name: bits} from gp_math.cuh's static_asserts."""
    with open(os.path.join(CSRC, "gp_math.cuh")) as fh:
        text = fh.read()
    pat = r"static_assert\(__builtin_bit_cast\(uint32_t, (\w+)\) == 0x([0-9A-Fa-f]{8})u"
    return {m.group(1): int(m.group(2), 16) for m in re.finditer(pat, text)}


def _bits(v):
    return int(np.float32(v).view(np.uint32))


def test_fast_loop_is_the_generator_output(tmp_path):
    shutil.copy(os.path.join(CSRC, "gen_fast.py"), tmp_path / "gen_fast.py")
    subprocess.run([sys.executable, str(tmp_path / "gen_fast.py")], check=True,
                   capture_output=True)
    with open(os.path.join(CSRC, "gp_fast.cuh")) as fh:
        committed = fh.read()
    assert (tmp_path / "gp_fast.cuh").read_text() == committed


def test_fitted_constants_match_the_pinned_bits():
    pinned = _pinned_bits()
    trig, log, exp = _load("fit_trig"), _load("fit_log"), _load("fit_exp")
    derived = {}
    for i, v in enumerate(trig.fit_sin_pi()):
        derived[f"kQ{i}"] = _bits(v)
    for name, v in zip(("kPiHi", "kPiMid", "kPiLo"), trig.split3(trig.PI)):
        derived[name] = _bits(v)
    for name, v in zip(("kPio2Hi", "kPio2Mid", "kPio2Lo"), trig.split3(trig.PI / 2)):
        derived[name] = _bits(v)
    S, C = trig.fit()
    for i, v in enumerate(S):
        derived[f"kS{i}"] = _bits(v)
    for i, v in enumerate(C):
        derived[f"kC{i}"] = _bits(v)
    for i, v in enumerate(log.fit()):
        derived[f"kLogP{i}"] = _bits(v)
    hi, lo = log.split_ln2()
    derived["kLn2Hi"], derived["kLn2Lo"] = _bits(hi), _bits(lo)
    for i, v in enumerate(exp.fit()):
        derived[f"kExpE{i + 1}"] = _bits(v)
    assert tuple(map(_bits, exp.split_ln2())) == (derived["kLn2Hi"], derived["kLn2Lo"])
    derived["kLog2e"] = _bits(exp.LOG2E)
    assert len(derived) == 35
    for name, bits in derived.items():
        assert pinned.get(name) == bits, (name, hex(bits), pinned.get(name))


def test_fast_loop_spells_the_pinned_constants():
    """gen_fast.py's bit patterns are the ones gp_math.cuh pins."""
    gen = _load("gen_fast")
    pinned = _pinned_bits()
    pairs = {"inv_pi": "kInvPi", "magic": "kRoundMagic", "pi_hi": "kPiHi", "pi_mid": "kPiMid",
             "pi_lo": "kPiLo", "q0": "kQ0", "q1": "kQ1", "q2": "kQ2", "q3": "kQ3",
             "trig_fast": "kTrigFast", "ln2_hi": "kLn2Hi", "ln2_lo": "kLn2Lo",
             "e1": "kExpE1", "e2": "kExpE2", "e3": "kExpE3", "e4": "kExpE4", "e5": "kExpE5",
             "e6": "kExpE6", "log2e": "kLog2e", "exp_fast": "kExpFast", "exp_inf": "kExpInf",
             "exp_zero": "kExpZero"}
    pairs.update({f"lp{i}": f"kLogP{i}" for i in range(8)})
    for key, name in pairs.items():
        assert gen.K[key] == pinned[name], (key, name)
