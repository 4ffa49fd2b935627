"""Derive the polynomial coefficients of gp_math.cuh's natural logarithm.

The evaluator's log runs on x = max(|a|, 0.001) > 0.  Write
x = 2^k m with m in [sqrt(1/2), sqrt(2)) (k from the exponent field after
subtracting the bit pattern of sqrt(1/2), m from the remaining bits), so
that f = m - 1 lies in [-0.2929, 0.4143] and is exact.  Then
    log x = k ln2 + log(1 + f),   log(1 + f) ~ f + f^2 P(f),
with P a degree-7 polynomial.  P minimises the maximum relative error of
log(1 + f) over the interval, found with Lawson's iteratively reweighted
least squares (C. L. Lawson, "Contributions to the theory of linear least
maximum approximation", 1961) on Chebyshev nodes in FP64, then rounded to
float32.  ln2 is split as LN2_HI + LN2_LO with LN2_HI holding 16
significant bits, so k * LN2_HI is exact for |k| <= 128.  The script
prints the coefficients and the float32-evaluated error (FMA emulated in
FP64) over a dense grid of x in [0.001, 3.4e38].

Run: python paper_2110_11226_gb300/csrc/fit_log.py
"""
from __future__ import annotations

import numpy as np

DEG = 7  # P(f) = P0 + P1 f + ... + P7 f^7
LO, HI = np.sqrt(0.5) - 1.0, np.sqrt(2.0) - 1.0


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
    f = LO + (HI - LO) * 0.5 * (1 + np.cos(np.pi * (k + 0.5) / len(k)))
    f = f[np.abs(f) > 1e-7]
    # (log1p f - f) / f^2 = P(f); relative error weight f^2 / log1p(f)
    A = np.stack([f ** i for i in range(DEG + 1)], axis=1)
    b = (np.log1p(f) - f) / f ** 2
    P = lawson(A, b, f ** 2 / np.log1p(f))
    return P.astype(np.float32)


def split_ln2():
    hi = np.float32(np.round(np.log(2.0) * 2.0 ** 15) / 2.0 ** 15)  # 16 significant bits
    lo = np.float32(np.log(2.0) - np.float64(hi))
    return hi, lo


def fma32(a, b, c):
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def log32(x, P, hi, lo):
    """The kernel's steps in float32 (FMA emulated in FP64), x >= 0.001 finite."""
    x = np.asarray(x, np.float32)
    i = x.view(np.int32).astype(np.int64)
    d = i - 0x3F3504F3
    k = d >> 23
    m = (i - (k << 23)).astype(np.int32).view(np.float32)
    f = np.float32(m - np.float32(1.0))
    kf = np.float32(k)
    p = np.full_like(f, P[DEG])
    for c in P[DEG - 1::-1]:
        p = fma32(p, f, c)
    y = np.float32(f * f)
    r = fma32(y, p, f)
    r = fma32(kf, lo, r)
    return fma32(kf, hi, r)


if __name__ == "__main__":
    P = fit()
    hi, lo = split_ln2()
    for i, v in enumerate(P):
        print(f"P{i} = {float(v)!r}f  // {int(v.view(np.uint32)):#010x}")
    print(f"LN2_HI = {float(hi)!r}f  // {int(hi.view(np.uint32)):#010x}")
    print(f"LN2_LO = {float(lo)!r}f  // {int(lo.view(np.uint32)):#010x}")
    # every float in [sqrt(1/2), 2 sqrt(2)) (the interval and one binade on),
    # then a log-spaced sweep of [0.001, 3.4e38]
    a = np.arange(np.float32(np.sqrt(0.5)).view(np.int32), np.float32(2 * np.sqrt(2.0)).view(np.int32),
                  dtype=np.int32).view(np.float32)
    b = np.exp(np.linspace(np.log(0.001), np.log(3.4e38), 4_000_001)).astype(np.float32)
    worst = 0.0
    for x in (a, b):
        got = log32(x, P, hi, lo).astype(np.float64)
        ref = np.log(x.astype(np.float64))
        ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
        worst = max(worst, float(np.max(np.abs(got - ref) / ulp)))
    print(f"max error over [0.001, 3.4e38] (float32 evaluation): {worst:.3f} ulp")
