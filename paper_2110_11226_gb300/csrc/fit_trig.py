"""Derive the polynomial coefficients of gp_math.cuh's sin/cos kernels.

On r in [-pi/4, pi/4]:
    sin r ~= r + r^3 (S0 + r^2 (S1 + r^2 (S2 + r^2 S3)))
    cos r ~= 1 + r^2 (-1/2 + r^2 (C0 + r^2 (C1 + r^2 (C2 + r^2 C3))))
The free coefficients minimise the maximum relative error, found with
Lawson's iteratively reweighted least squares (C. L. Lawson, "Contributions
to the theory of linear least maximum approximation", 1961) on Chebyshev
nodes in FP64, then rounded to float32.  The script also prints the
float32-evaluated error (FMA emulated in FP64) over a dense grid.

Run: python paper_2110_11226_gb300/csrc/fit_trig.py
"""
from __future__ import annotations

import numpy as np


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


def f32(x):
    return np.float32(x)


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
    S, C = fit()
    for i, v in enumerate(S):
        print(f"S{i} = {v!r}f  // {v.view(np.uint32):#010x}")
    for i, v in enumerate(C):
        print(f"C{i} = {v!r}f  // {v.view(np.uint32):#010x}")
    grid = np.linspace(-np.pi / 4, np.pi / 4, 200001).astype(np.float32)
    es = max(abs(float(eval_sin(x, S)) - np.sin(np.float64(x))) / np.spacing(np.float32(abs(np.sin(np.float64(x))) or 1e-30))
             for x in grid[::7] if x != 0)
    ec = max(abs(float(eval_cos(x, C)) - np.cos(np.float64(x))) / np.spacing(np.float32(np.cos(np.float64(x))))
             for x in grid[::7])
    print(f"max error on [-pi/4, pi/4] (float32 evaluation): sin {es:.3f} ulp, cos {ec:.3f} ulp")
