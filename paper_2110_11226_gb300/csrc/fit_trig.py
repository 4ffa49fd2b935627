"""Derive the polynomial coefficients of gp_math.cuh's sin, cos and tan.

sin and cos: one odd polynomial on r in [-pi/2, pi/2] (with 0.05% slack
for a rounded quotient),
    sin r ~= r + r^3 (Q0 + r^2 (Q1 + r^2 (Q2 + r^2 Q3))),
after the reduction r = x - j pi (sin) or x - (j + 1/2) pi (cos) against
a three-part split of pi, so that sin x = +-sin r and cos x = -+sin r.
tan: the quotient of
    sin r ~= r + r^3 (S0 + r^2 (S1 + r^2 (S2 + r^2 S3)))
    cos r ~= 1 + r^2 (-1/2 + r^2 (C0 + r^2 (C1 + r^2 (C2 + r^2 C3))))
on r in [-pi/4, pi/4] after a reduction by pi/2.  The free coefficients
minimise the maximum relative error, found with Lawson's iteratively
reweighted least squares (C. L. Lawson, "Contributions to the theory of
linear least maximum approximation", 1961) on Chebyshev nodes in FP64,
then rounded to float32.  The three-part splits of pi and pi/2 come from a
50-digit value of pi.  The script prints the coefficients and the
float32-evaluated error of sin and cos (FMA emulated in FP64) over |x| <
65536, the floats nearest the multiples of pi/2 included.

Run: python paper_2110_11226_gb300/csrc/fit_trig.py
"""
from __future__ import annotations

from decimal import Decimal, getcontext

import numpy as np

getcontext().prec = 60
PI = Decimal("3.14159265358979323846264338327950288419716939937510")


def lawson(A, b, w0, iters=200):
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
    hi = np.pi / 4
    k = np.arange(4000)
    r = hi * 0.5 * (1 + np.cos(np.pi * (k + 0.5) / len(k)))  # Chebyshev nodes on (0, hi)
    r = r[r > 1e-6]
    r2 = r * r
    # sin: (sin r - r) / r^3 = S0 + S1 r^2 + S2 r^4 + S3 r^6, relative error weight r^3/sin r
    A = np.stack([r2 ** i for i in range(4)], axis=1)
    b = (np.sin(r) - r) / r ** 3
    S = lawson(A, b, r ** 3 / np.sin(r))
    # cos: (cos r - 1 + r^2/2) / r^4 = C0 + C1 r^2 + C2 r^4 + C3 r^6
    b = (np.cos(r) - 1 + r2 / 2) / r2 ** 2
    C = lawson(A, b, r2 ** 2 / np.cos(r))
    return S.astype(np.float32), C.astype(np.float32)


def split3(v: Decimal):
    """v = HI + MID + LO, each the float32 nearest what remains"""
    parts = []
    for _ in range(3):
        f = np.float32(float(v))
        parts.append(f)
        v -= Decimal(float(f))
    return parts


def fit_sin_pi(terms=4, span=1.0005):
    hi = np.pi / 2 * span
    k = np.arange(8000)
    r = hi * 0.5 * (1 + np.cos(np.pi * (k + 0.5) / len(k)))
    r = r[r > 1e-6]
    A = np.stack([(r * r) ** i for i in range(terms)], axis=1)
    return lawson(A, (np.sin(r) - r) / r ** 3, r ** 3 / np.sin(r)).astype(np.float32)


INV_PI = np.float32(1.0 / np.pi)
MAGIC = np.float32(12582912.0)


def sincos32(x, kind, Q, pi3):
    """The kernel's steps in float32 (FMA emulated in FP64), |x| < 65536"""
    x = np.asarray(x, np.float32)
    half = np.float32(0.5 * kind)
    t1 = fma32(x, INV_PI, -half)
    jm = np.float32(t1 + MAGIC)
    jj = np.float32(jm - MAGIC)
    jh = np.float32(jj + half)
    r = x
    for part in pi3:
        r = fma32(jh, -part, r)
    s = np.float32(r * r)
    p = np.full_like(s, Q[-1])
    for c in Q[-2::-1]:
        p = fma32(p, s, c)
    v = fma32(p, np.float32(s * r), r)
    q = (jm.view(np.int32).astype(np.int64) - 0x4B400000) + kind
    return np.where((q & 1) == 1, -v, v).astype(np.float32)


def fma32(a, b, c):
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def eval_sin(r, S):
    r = np.float32(r)
    s = np.float32(r * r)
    p = S[3]
    for c in (S[2], S[1], S[0]):
        p = fma32(p, s, c)
    return fma32(p, np.float32(s * r), r)


def eval_cos(r, C):
    r = np.float32(r)
    s = np.float32(r * r)
    p = C[3]
    for c in (C[2], C[1], C[0]):
        p = fma32(p, s, c)
    p = fma32(p, s, np.float32(-0.5))
    return fma32(p, s, np.float32(1.0))


if __name__ == "__main__":
    Q = fit_sin_pi()
    pi3 = split3(PI)
    for i, v in enumerate(Q):
        print(f"Q{i} = {float(v)!r}f  // {int(v.view(np.uint32)):#010x}")
    for name, v in zip(("PI_HI", "PI_MID", "PI_LO"), pi3):
        print(f"{name} = {float(v)!r}f  // {int(v.view(np.uint32)):#010x}")
    for name, v in zip(("PIO2_HI", "PIO2_MID", "PIO2_LO"), split3(PI / 2)):
        print(f"{name} = {float(v)!r}f  // {int(v.view(np.uint32)):#010x}")
    S, C = fit()
    for i, v in enumerate(S):
        print(f"S{i} = {float(v)!r}f  // {int(v.view(np.uint32)):#010x}")
    for i, v in enumerate(C):
        print(f"C{i} = {float(v)!r}f  // {int(v.view(np.uint32)):#010x}")
    x = np.concatenate([np.linspace(-65536, 65536, 8_000_001).astype(np.float32),
                        np.linspace(-20, 20, 4_000_001).astype(np.float32)])
    near = (np.arange(-41000, 41000) * np.pi / 2).astype(np.float32)
    x = np.concatenate([x, near, np.nextafter(near, np.float32(np.inf)),
                        np.nextafter(near, np.float32(-np.inf))])
    x = x[np.abs(x) < 65536]
    for kind, name in ((0, "sin"), (1, "cos")):
        got = sincos32(x, kind, Q, pi3).astype(np.float64)
        ref = np.sin(x.astype(np.float64)) if kind == 0 else np.cos(x.astype(np.float64))
        ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
        print(f"max error of {name} over |x| < 65536 (float32 evaluation): "
              f"{np.max(np.abs(got - ref) / ulp):.3f} ulp")
