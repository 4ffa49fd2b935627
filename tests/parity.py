"""Parity helpers: compare GPU results with the FP64 oracle.

Per point (tolerance 1e-5 relative, FP32 evaluation against FP64):
  * the oracle gives, for every row, the FP64 value v, a first-order bound e
    on the error of any FP32 evaluation whose library functions err by at
    most ULPS units in the last place, and flags (1 = a protected
    operator's threshold test may decide differently in FP32, 2 = a value
    leaves the float range);
  * "ok" rows (no flag, e <= v/4 * 1e-5) must satisfy |gpu - v| <= 1e-5 |v|;
  * "conditioning" rows (no flag, larger e) must satisfy |gpu - v| <= 1.5 e
    + 1e-5 |v| -- FP32 cannot meet 1e-5 there, the bound says by how much;
  * flagged rows are counted, not compared.
Fitness (tolerance 1e-4 relative): programs whose rows are all unflagged
and whose propagated bound is below 1e-4/4 of the fitness must match within
1e-4; the others must stay within the propagated bound and are counted.
"""
from __future__ import annotations

import dataclasses

import numpy as np

import oracle

ULPS = 4.0          # CUDA: sinf/cosf/expf 2 ulp, tanf 4, logf/log1pf 1
REL_POINT = 1e-5
REL_FIT = 1e-4


@dataclasses.dataclass
class PointStats:
    rows: int
    ok: int
    conditioning: int
    flagged: int


def check_points(gpu, nodes, off, X, row0=0, n_eval=None):
    gpu = np.asarray(gpu, np.float64)
    v, e, fl = oracle.predict_bound(nodes, off, X, row0=row0, n_eval=n_eval, ulps_fn=ULPS)
    assert gpu.shape == v.shape
    unfl = fl == 0
    tight = unfl & (e <= 0.25 * REL_POINT * np.abs(v))
    cond = unfl & ~tight
    with np.errstate(invalid="ignore"):
        err = np.abs(gpu - v)
    bad_ok = tight & ~(err <= REL_POINT * np.abs(v))
    assert not bad_ok.any(), _report(bad_ok, gpu, v, e)
    bad_c = cond & ~(err <= 1.5 * e + REL_POINT * np.abs(v))
    # a NaN FP64 value (e.g. sin(inf)) must be NaN on the GPU as well
    both_nan = np.isnan(gpu) & np.isnan(v)
    bad_c &= ~both_nan
    assert not bad_c.any(), _report(bad_c, gpu, v, e)
    return PointStats(int(v.size), int(tight.sum()), int(cond.sum()), int((~unfl).sum())), (v, e, fl)


def _report(mask, gpu, v, e):
    idx = np.argwhere(mask)[:5]
    return "mismatch at " + "; ".join(
        f"{tuple(i)}: gpu={gpu[tuple(i)]!r} fp64={v[tuple(i)]!r} bound={e[tuple(i)]!r}" for i in idx)


def fitness_bound(metric, v, e, y, w):
    """Propagate per-row FP32 bounds e into a bound on the weighted metric."""
    y = y.astype(np.float64)
    wv = np.ones_like(y) if w is None else w.astype(np.float64)
    sw = wv.sum()
    with np.errstate(all="ignore"):
        if metric == "mae" or metric == "logloss":  # |dl/dp| <= 1
            b = (e * wv).sum(axis=1) / sw
        else:
            d = np.abs(v - y[None, :])
            b = ((2 * d * e + e * e) * wv).sum(axis=1) / sw
    return b


@dataclasses.dataclass
class FitStats:
    programs: int
    strict: int
    conditioning: int
    flagged: int
    max_rel_strict: float


def _bound_terms(nodes, off, X, y, w, metric, row0, n_eval, block):
    """Per program: the propagated FP32 bound on the metric's mean (before
    the root of RMSE), whether any row is flagged, and the largest and the
    total weighted row loss, over rows [row0, row0 + n_eval) taken in blocks
    of rows (memory stays bounded at full size)."""
    P = len(off) - 1
    wv_all = None if w is None else w.astype(np.float64)
    sw = float(n_eval) if wv_all is None else wv_all[row0:row0 + n_eval].sum()
    bsum = np.zeros(P)
    flag = np.zeros(P, bool)
    lmax = np.zeros(P)
    lsum = np.zeros(P)
    mse_metric = "mse" if metric == "rmse" else metric
    for r in range(row0, row0 + n_eval, block):
        m = min(block, row0 + n_eval - r)
        v, e, fl = oracle.predict_bound(nodes, off, X, row0=r, n_eval=m, ulps_fn=ULPS)
        ys = y[r:r + m]
        ws = None if wv_all is None else wv_all[r:r + m]
        wsum = float(m) if ws is None else ws.sum()
        bsum += fitness_bound(mse_metric, v, e, ys, ws) * wsum
        flag |= (fl != 0).any(axis=1)
        with np.errstate(all="ignore"):
            yy = ys.astype(np.float64)[None, :]
            if metric == "mae":
                rl = np.abs(v - yy)
            elif metric == "logloss":
                rl = np.abs(v) + np.log(2.0)
            else:
                rl = (v - yy) ** 2
            wl = rl if ws is None else rl * ws[None, :]
            lmax = np.fmax(lmax, np.nanmax(wl, axis=1))
            lsum += np.nansum(wl, axis=1)
    return bsum / sw, flag, lmax, lsum


def check_fitness(gpu_fit, nodes, off, X, y, w, metric, row0=0, n_eval=None, block=1 << 18):
    """Fitness against the FP64 oracle: programs whose rows are all
    unflagged and whose propagated FP32 bound is below a quarter of 1e-4 of
    the fitness ("strict") must match within 1e-4 relative; the others
    ("conditioning") within 1.5 x the bound + 1e-4; flagged ones (a
    protected decision may flip, a value or loss leaves the float range)
    are counted.  The bound is accumulated over blocks of rows."""
    gpu_fit = np.asarray(gpu_fit, np.float64)
    n_eval = X.shape[1] - row0 if n_eval is None else n_eval
    f64, st = oracle.fitness(nodes, off, X, y, w, metric, row0=row0, n_eval=n_eval)
    b, fl_any, lmax, lsum = _bound_terms(nodes, off, X, y, w, metric, row0, n_eval, block)
    f_cmp = f64
    g_cmp = gpu_fit
    if metric == "rmse":  # compare squares: the bound is on the MSE
        f_cmp = f64 ** 2
        g_cmp = gpu_fit ** 2
    # FP32 range of the loss itself: a weighted row loss, or the sum of a
    # chunk's losses, beyond the float range is +inf on the GPU while the
    # FP64 oracle stays finite (all losses are >= 0, so the total bounds
    # every partial sum)
    FMAX = float(np.finfo(np.float32).max)
    loss_range = (lmax > 0.5 * FMAX) | (lsum > 0.5 * FMAX)
    flagged = fl_any | (st != 0) | loss_range
    with np.errstate(invalid="ignore"):
        strict = ~flagged & np.isfinite(f64) & (b <= 0.25 * REL_FIT * np.abs(f_cmp))
        rel = np.abs(gpu_fit - f64) / np.maximum(np.abs(f64), 1e-300)
        strict_ok = ~strict | (rel <= REL_FIT) | (np.abs(gpu_fit - f64) <= 1e-12)
    assert strict_ok.all(), f"fitness mismatch: {np.argwhere(~strict_ok)[:5].ravel()} rel={rel[~strict_ok][:5]}"
    cond = ~flagged & ~strict
    with np.errstate(invalid="ignore"):
        cond_ok = ~cond | (np.abs(g_cmp - f_cmp) <= 1.5 * b + REL_FIT * np.abs(f_cmp)) | \
            (np.isinf(g_cmp) & np.isinf(f_cmp))
    assert cond_ok.all(), f"conditioning fitness beyond bound: {np.argwhere(~cond_ok)[:5].ravel()}"
    # status: malformed programs are NaN on both sides
    assert np.all(np.isnan(gpu_fit[st != 0]))
    mr = float(np.max(rel[strict])) if strict.any() else 0.0
    return FitStats(len(f64), int(strict.sum()), int(cond.sum()), int(flagged.sum()), mr), f64


def check_pearson(gpu_fit, nodes, off, X, y, w):
    """Weighted Pearson fitness |r| against the FP64 oracle.

    A per-row FP32 error e moves the centred prediction vector by at most
    ||e||_w, and |r| is the cosine of the angle between the centred
    prediction and target vectors, so |d|r|| <= 2 ||e||_w / sd_w(p); the
    FP32 accumulation of the shifted moment sums adds a relative error of a
    few ulp of E_w[(p - p0)^2] / var_w(p) (p0 = the value on row 0, the
    evaluator's shift; 32 ulp of FP32 covers the 8-row plain sums inside
    the compensated per-lane sums).  Programs with flagged rows, or whose squared
    deviations leave the float range, are counted, not compared."""
    gpu_fit = np.asarray(gpu_fit, np.float64)
    f64, st = oracle.fitness(nodes, off, X, y, w, "pearson")
    v, e, fl = oracle.predict_bound(nodes, off, X, ulps_fn=ULPS)
    wv = np.ones(v.shape[1]) if w is None else w.astype(np.float64)
    sw = wv.sum()
    FMAX = float(np.finfo(np.float32).max)
    with np.errstate(all="ignore"):
        mean = (v * wv).sum(axis=1) / sw
        var = (((v - mean[:, None]) ** 2) * wv).sum(axis=1) / sw
        dev0 = (((v - v[:, :1]) ** 2) * wv)
        ew = np.sqrt((e * e * wv).sum(axis=1) / sw)
        b = 2.0 * ew / np.sqrt(var) + 2e-6 * (dev0.sum(axis=1) / sw) / var
        rng_flag = (np.nanmax(dev0, axis=1) > 0.5 * FMAX) | (dev0.sum(axis=1) > 0.5 * FMAX) | \
            ~np.isfinite(v).all(axis=1)
    flagged = (fl != 0).any(axis=1) | (st != 0) | rng_flag
    with np.errstate(invalid="ignore"):
        strict = ~flagged & np.isfinite(f64) & (var > 0) & (b <= 0.25 * REL_FIT * np.abs(f64))
        err = np.abs(gpu_fit - f64)
        strict_ok = ~strict | (err <= REL_FIT * np.abs(f64)) | (err <= 1e-12)
    assert strict_ok.all(), f"pearson mismatch: {np.argwhere(~strict_ok)[:5].ravel()}"
    cond = ~flagged & ~strict
    with np.errstate(invalid="ignore"):
        cond_ok = ~cond | (err <= 1.5 * b + REL_FIT * np.abs(f64)) | (np.isnan(b) & (var == 0))
        # a program constant in FP64 is constant in FP32 too when the
        # constant does not depend on the row: both give exactly 0
        zero_ok = ~(cond & (var == 0)) | (gpu_fit == 0) | (b > 0)
    assert cond_ok.all(), f"pearson beyond bound: {np.argwhere(~cond_ok)[:5].ravel()}"
    assert zero_ok.all()
    assert np.all(np.isnan(gpu_fit[st != 0]))
    mr = float(np.max(err[strict] / np.abs(f64[strict]))) if strict.any() else 0.0
    return FitStats(len(f64), int(strict.sum()), int(cond.sum()), int(flagged.sum()), mr), f64


def check_fitness_sampled(gpu_fit, nodes, off, X, y, w, metric):
    """Full-size fitness of sampled programs: check_fitness over every row,
    its bound accumulated in blocks.  Returns (strict, conditioning,
    flagged) counts."""
    st, _ = check_fitness(gpu_fit, nodes, off, X, y, w, metric)
    return st.strict, st.conditioning, st.flagged
