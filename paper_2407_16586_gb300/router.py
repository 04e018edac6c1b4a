"""Training pipeline of the learned block router.

Samples quartet tiles of seeded training clusters (fp64 and fp32 evaluation
of the same tiles, no reduction), trains the MLP on the GPU, and calibrates
two constants on held-out tiles:

* margin: the 99th percentile of (log10 true contribution - prediction), so
  10^(prediction + margin) is rarely below the tile's true contribution;
* eps_rel: the 99th percentile of the fp32 error of a tile's contribution
  relative to the contribution.

TG_MIXED_LEARNED then sends tiles to fp32 in increasing order of
e_t = eps_rel * 10^(prediction + margin) while sum e_t^2 <= mixed_tol^2
(mixed_tol defaults to 1e-6 Ha/bohr).

Both percentiles bound single tiles, so the summed estimate overstates the
error of the routed set by orders of magnitude.  calibrate_budget() then
measures the whole route: on held-out molecules it runs the mixed path
against fp64 while lowering the margin in steps of 0.25 (log10), and keeps
the lowest margin whose largest max|dg| stays within mixed_tol / safety.
The single safety factor (default 2) covers the spread of the error between
molecules: at a fixed margin the measured errors of the budget molecules
differ by a factor recorded in the calibration log (spread), and the
factor is chosen at least as large as that spread."""
from __future__ import annotations

import numpy as np

import paper_2407_16586_gb300 as tg


def collect(systems, stride=40, cap=200000, screen_tol=1e-10):
    Xs, ys, es = [], [], []
    for s in systems:
        b = tg.Basis(s)
        X, y, e = b.tile_samples(s["pairs"], stride=stride, cap=cap, screen_tol=screen_tol)
        b.close()
        Xs.append(X)
        ys.append(y)
        es.append(e)
    return np.concatenate(Xs), np.concatenate(ys), np.concatenate(es)


def fit(X, y, e, seed=7, epochs=400, lr=1e-2, q=0.9, holdout=0.2, floor=-20.0):
    """Train on (1 - holdout) of the tiles and calibrate on the rest.
    Tiles whose contribution is below 10^floor carry no information about
    routing and are clipped to the floor."""
    y = np.maximum(y, floor).astype(np.float32)
    rng = np.random.default_rng(seed)
    idx = rng.permutation(len(y))
    nh = max(1, int(holdout * len(y)))
    hold, tr = idx[:nh], idx[nh:]
    r = tg.Router(seed=seed)
    hist = r.train(X[tr], y[tr], epochs=epochs, lr=lr, q=q)
    pred = r.predict(X[hold])
    margin = float(max(0.0, np.quantile(y[hold] - pred, 0.99)))
    rel = 10.0 ** (e - y)
    keep = y > floor + 1
    eps_rel = float(np.quantile(rel[keep], 0.99)) if keep.any() else 1e-5
    r.set(calib=[margin, eps_rel, 1.0])
    info = dict(n_train=len(tr), n_hold=nh, loss_first=float(hist[0]), loss_last=float(hist[-1]), margin=margin,
                eps_rel=eps_rel, resid_hold_mean=float(np.mean(y[hold] - pred)))
    return r, info


def calibrate_budget(r, systems, mixed_tol=1e-6, safety=2.0, step=0.25, max_steps=32, screen_tol=1e-10,
                     shards=None):
    """Lower the router's margin while the measured max|dg| of TG_MIXED_LEARNED
    against TG_FP64 over ``systems`` stays <= mixed_tol / safety.  ``shards``
    (optional, one (rank, nranks) or None per system) evaluates a pair-key
    shard of a system, so that a full-size system can sit in the budget set.
    Returns a list of (margin, max error, fp32 quartet fraction, spread) for
    every margin tried; spread = largest / smallest per-system error."""
    params, mu, sd, calib = r.get()
    margin0, eps_rel = float(calib[0]), float(calib[1])
    shards = shards or [None] * len(systems)
    runs = []
    for s, sh in zip(systems, shards):
        b = tg.Basis(s)
        kw = dict(rank=sh[0], nranks=sh[1]) if sh else {}
        g64, _ = b.grad2e(s["pairs"], screen_tol=screen_tol, **kw)
        runs.append((b, s, g64, kw))
    best, log = margin0, []
    for k in range(max_steps + 1):
        m = margin0 - step * k
        r.set(calib=[m, eps_rel, 1.0])
        errs, q32, q = [], 0, 0
        for b, s, g64, kw in runs:
            g, st = b.grad2e(s["pairs"], screen_tol=screen_tol, precision=tg.TG_MIXED_LEARNED, router=r,
                             mixed_tol=mixed_tol, **kw)
            errs.append(float(np.abs(g - g64).max()))
            q32 += st["fp32_quartets"]
            q += st["quartets"]
        err = max(errs)
        nz = [e for e in errs if e > 0]
        spread = max(nz) / min(nz) if nz else 1.0
        log.append((m, err, q32 / max(q, 1), spread))
        if err > mixed_tol / safety:
            break
        best = m
    r.set(calib=[best, eps_rel, 1.0])
    for b, _, _, _ in runs:
        b.close()
    return log
