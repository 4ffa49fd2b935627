"""Derive the polynomial coefficients of gp_math.cuh's exponential.

For |x| < 87 the evaluator computes e^x as 2^j e^r: j is x log2(e) rounded
to the nearest integer (in the FMA pipe, by adding 1.5 * 2^23), and
r = x - j ln2 in two fused multiply-adds against LN2_HI + LN2_LO (LN2_HI
with 16 significant bits, so j * LN2_HI is exact), the reduction of W. J.
Cody and W. Waite, "Software Manual for the Elementary Functions", 1980.
On r in [-0.35, 0.35] (ln2 / 2 plus the slack of a rounded j)
    e^r ~ 1 + r (E1 + r (E2 + r (E3 + r (E4 + r (E5 + r E6)))))
with E1..E6 minimising the maximum relative error (Lawson's iteratively
reweighted least squares, C. L. Lawson, 1961, on Chebyshev nodes in FP64,
then rounded to float32).  2^j (-126 <= j <= 126 for |x| < 87) is built
in the exponent field and the product is one rounding.  Outside |x| < 87
(and for NaN) the evaluator calls CUDA's expf instead.

Run: python paper_2110_11226_gb300/csrc/fit_exp.py
"""
from __future__ import annotations

import numpy as np

R = 0.35
DEG = 6


def lawson(A, b, w0, iters=300):
    """Minimise max |w0 * (A c - b)| by Lawson's reweighting."""
    n = A.shape[0]
    lam = np.full(n, 1.0 / n)
    c = None
    for _ in range(iters):
        W = np.sqrt(lam) * w0
        c, *_ = np.linalg.lstsq(A * W[:, None], b * W, rcond=None)
        e = np.abs(w0 * (A @ c - b))
        lam = lam * e
        s = lam.sum()
        if s == 0:
            break
        lam /= s
    return c


def fit():
    k = np.arange(6000)
    r = R * np.cos(np.pi * (k + 0.5) / len(k))
    r = r[np.abs(r) > 1e-9]
    # (e^r - 1) / r = E1 + E2 r + ... + E6 r^5; relative error weight r / e^r
    A = np.stack([r ** i for i in range(DEG)], axis=1)
    b = np.expm1(r) / r
    E = lawson(A, b, r / np.exp(r))
    return E.astype(np.float32)


def split_ln2():
    hi = np.float32(np.round(np.log(2.0) * 2.0 ** 15) / 2.0 ** 15)  # 16 significant bits
    lo = np.float32(np.log(2.0) - np.float64(hi))
    return hi, lo


LOG2E = np.float32(1.0 / np.log(2.0))
MAGIC = np.float32(12582912.0)


def fma32(a, b, c):
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def exp32(x, E, hi, lo):
    """The kernel's steps in float32 (FMA emulated in FP64), |x| < 87."""
    x = np.asarray(x, np.float32)
    jm = fma32(x, LOG2E, MAGIC)
    jf = np.float32(jm - MAGIC)
    r = fma32(jf, -hi, x)
    r = fma32(jf, -lo, r)
    p = np.full_like(r, E[DEG - 1])
    for c in E[DEG - 2::-1]:
        p = fma32(p, r, c)
    p = fma32(p, r, np.float32(1.0))
    j = jm.view(np.int32).astype(np.int64) - 0x4B400000
    s = ((j + 127) << 23).astype(np.int32).view(np.float32)
    return np.float32(p * s)


if __name__ == "__main__":
    E = fit()
    hi, lo = split_ln2()
    for i, v in enumerate(E):
        print(f"E{i + 1} = {float(v)!r}f  // {int(v.view(np.uint32)):#010x}")
    print(f"LN2_HI = {float(hi)!r}f  // {int(hi.view(np.uint32)):#010x}")
    print(f"LN2_LO = {float(lo)!r}f  // {int(lo.view(np.uint32)):#010x}")
    print(f"LOG2E = {float(LOG2E)!r}f  // {int(LOG2E.view(np.uint32)):#010x}")
    x = np.linspace(-87.0, 87.0, 8_000_001).astype(np.float32)
    x = x[np.abs(x) < 87.0]
    x = np.concatenate([x, np.arange(np.float32(-1).view(np.int32), np.float32(-0.0).view(np.int32),
                                     977, dtype=np.int32).view(np.float32)])
    got = exp32(x, E, hi, lo).astype(np.float64)
    ref = np.exp(x.astype(np.float64))
    ulp = np.spacing(ref.astype(np.float32)).astype(np.float64)
    print(f"max error over |x| < 87 (float32 evaluation): {np.max(np.abs(got - ref) / ulp):.3f} ulp")
