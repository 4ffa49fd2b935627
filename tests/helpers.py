"""Small helpers shared by the tests (parsing hand-written programs, tolerances)."""
from __future__ import annotations

import os

import numpy as np

from paper_2110_11226_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def parse_prefix(text: str):
    """'sub x0 0.5' -> list of (op, feat, c) nodes in prefix order."""
    out = []
    for tok in text.split():
        if tok in synth.OP:
            out.append((synth.OP[tok], 0, 0.0))
        elif tok.startswith("x") and tok[1:].isdigit():
            out.append((synth.OP["var"], int(tok[1:]), 0.0))
        else:
            out.append((synth.OP["const"], 0, float(np.float32(float(tok)))))
    return out


def read_table(name: str):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([c.strip() for c in line.split(";")])
    return rows


def pack(programs):
    return synth.pack(programs)
