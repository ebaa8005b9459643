"""Calibrate the epsilon of each named workload with the CPU oracle (test infrastructure).

Writes paper_1812_07607_gb300/workload_eps.json. The paper states no epsilon
for its image-matching queries (Sec. 6.2), so each workload fixes its
selectivity instead and this script turns that into a value:

  * rxs_histograms_2k: every one of the 4,000,000 canonical distances is
    computed; eps^2 sits in the gap after the 4,000th smallest (0.1%
    selectivity).
  * self_clustered_262k: 512 seeded rows against all 262,144 rows; eps^2 sits
    in the gap that makes the mean number of other rows within eps equal 20.
  * rxs_unit_mixture_1m: 64 seeded R rows against all of S; mean 10 per row.
  * hist_clustered_64k (L1 / chi-square self-joins): 256 seeded rows against
    all 65,536 rows per metric; the threshold sits in the gap that gives a mean of
    20 other rows per row (these distances are not squared, so the threshold is
    the gap's midpoint itself).
  * tracked_objects_262k (pruned join): 256 seeded rows against all 262,144 rows;
    eps sits in the gap that gives a mean of 100 other rows within eps per row.
  * batch_store_2m / serve_store_4m (request workloads): 256 fresh query rows against a
    seeded 65,536-row sample of the store; the pooled distances give a
    (selectivity, eps) table, selectivity = the fraction of store rows within eps.

eps is then placed so that fl(eps*eps) lies strictly inside the chosen gap of
the sampled canonical distances (the gap's midpoint), keeping every sampled
distance away from the threshold. Every distance comes from the oracle.

    python -m oracle.calibrate_eps [name ...]
"""

from __future__ import annotations

import json
import math
import multiprocessing as mp
import os
import sys

import numpy as np

import oracle
from paper_1812_07607_gb300 import workloads as W

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1812_07607_gb300", "workload_eps.json")


def _block_smallest(args):
    R, S, keep, excl = args[:4]
    metric = args[4] if len(args) > 4 else 0
    D = oracle.default().dist_block(R, S) if metric == 0 else oracle.default().hist_dist_block(R, S, metric)
    if excl is not None:
        D[np.arange(D.shape[0]), excl] = np.inf
    keep = min(keep, D.shape[1] - 1)
    return np.sort(np.partition(D, keep, axis=1)[:, :keep + 1], axis=1)


def smallest_per_row(R, S, keep, excl=None, procs=None, block=8, metric=0):
    procs = procs or min(8, os.cpu_count() or 1)
    jobs = []
    for r0 in range(0, R.shape[0], block):
        r1 = min(R.shape[0], r0 + block)
        jobs.append((R[r0:r1], S, keep, None if excl is None else excl[r0:r1], metric))
    with mp.get_context("spawn").Pool(procs) as pool:
        parts = pool.map(_block_smallest, jobs)
    return np.concatenate(parts, axis=0)


def thr_in_gap(sorted_vals: np.ndarray, rank: int) -> float:
    """An unsquared threshold strictly between sorted_vals[rank-1] and the next larger value."""
    a = sorted_vals[rank - 1]
    b = sorted_vals[np.searchsorted(sorted_vals, a, side="right")]
    t = 0.5 * (a + b)
    if not (a < t < b):
        raise RuntimeError(f"gap too narrow at rank {rank}: {a!r} {b!r}")
    return t


def eps_in_gap(sorted_vals: np.ndarray, rank: int) -> float:
    """eps with fl(eps^2) strictly between sorted_vals[rank-1] and the next larger value."""
    a = sorted_vals[rank - 1]
    b = sorted_vals[np.searchsorted(sorted_vals, a, side="right")]
    mid = 0.5 * (a + b)
    eps = math.sqrt(mid)
    e2 = eps * eps
    if not (a < e2 < b):
        raise RuntimeError(f"gap too narrow at rank {rank}: {a!r} {b!r}")
    return eps


def calibrate(name: str) -> tuple[str, float, dict]:
    if name == "rxs_histograms_2k":
        wl = W.rxs_histograms_2k(eps=0.0)
        D = oracle.default().dist_block(wl.R, wl.S)
        vals = np.sort(D.ravel())
        target = wl.pairs // 1000
        eps = eps_in_gap(vals, target)
        key = f"rxs_histograms_2k:{W.SEED_BASE + 0}:2000:64"
        return key, eps, {"pairs_at_eps": int((vals <= eps * eps).sum())}
    if name == "self_clustered_262k":
        wl = W.self_clustered_262k(eps=0.0)
        g = W.rng(W.SEED_BASE + 101)
        rows = np.sort(g.choice(wl.R.shape[0], size=512, replace=False))
        sm = smallest_per_row(wl.R[rows], wl.R, keep=1600, excl=rows)
        vals = np.sort(sm.ravel())
        target = 20 * len(rows)
        eps = eps_in_gap(vals, target)
        key = f"self_clustered_262k:{W.SEED_BASE + 1}:262144:128:8192"
        per_row = (sm <= eps * eps).sum(axis=1)
        # selectivity -> eps table (batch / serving request mixes): pooled quantiles of the
        # sampled rows' canonical distances, s = matches per row / (N - 1)
        table = []
        for sel in np.geomspace(1e-5, 5.5e-3, 40):
            rank = int(round(sel * (wl.R.shape[0] - 1) * len(rows)))
            table.append([float(sel), eps_in_gap(vals, max(1, rank))])
        extra = {"self_clustered_262k:selectivity_eps": table}
        return key, eps, {"sample_rows": 512, "mean_matches": float(per_row.mean()),
                          "max_row_kept_fill": float((sm[:, -1] <= eps * eps).mean()), "extra": extra}
    if name == "rxs_unit_mixture_1m":
        wl = W.rxs_unit_mixture_1m(eps=0.0)
        g = W.rng(W.SEED_BASE + 102)
        rows = np.sort(g.choice(wl.R.shape[0], size=64, replace=False))
        sm = smallest_per_row(wl.R[rows], wl.S, keep=200)
        vals = np.sort(sm.ravel())
        eps = eps_in_gap(vals, 10 * len(rows))
        key = f"rxs_unit_mixture_1m:{W.SEED_BASE + 2}:1048576:512:4096"
        per_row = (sm <= eps * eps).sum(axis=1)
        return key, eps, {"sample_rows": 64, "mean_matches": float(per_row.mean())}
    if name == "tracked_objects_262k":
        wl = W.tracked_objects_262k(eps=0.0)
        g = W.rng(W.SEED_BASE + 108)
        rows = np.sort(g.choice(wl.R.shape[0], size=256, replace=False))
        sm = smallest_per_row(wl.R[rows], wl.R, keep=1000, excl=rows)
        vals = np.sort(sm.ravel())
        eps = eps_in_gap(vals, 100 * len(rows))
        key = f"tracked_objects_262k:{W.SEED_BASE + 7}:262144:128:256"
        return key, eps, {"sample_rows": 256, "mean_matches": float((sm <= eps * eps).sum(axis=1).mean())}
    if name == "hist_clustered_64k":
        X, _ = W.hist_clustered_64k()
        g = W.rng(W.SEED_BASE + 106)
        rows = np.sort(g.choice(X.shape[0], size=256, replace=False))
        extra = {}
        for mname, metric in (("l1", oracle.METRIC_L1), ("chi2", oracle.METRIC_CHI2)):
            sm = smallest_per_row(X[rows], X, keep=400, excl=rows, metric=metric)
            vals = np.sort(sm.ravel())
            extra[f"hist_clustered_64k:{mname}:{W.SEED_BASE + 6}"] = thr_in_gap(vals, 20 * len(rows))
        return None, None, {"extra": extra}
    if name in ("batch_store_2m", "serve_store_4m"):
        st = getattr(W, name)()
        g = W.rng(W.SEED_BASE + 104)
        cols = np.sort(g.choice(st.X.shape[0], size=65536, replace=False))
        Q = st.queries(256, W.SEED_BASE + 105)
        sm = smallest_per_row(Q, np.ascontiguousarray(st.X[cols]), keep=2000)
        vals = np.sort(sm.ravel())
        table = []
        for sel in np.geomspace(1e-5, 5.5e-3, 40):
            rank = int(round(sel * len(cols) * Q.shape[0]))
            table.append([float(sel), eps_in_gap(vals, max(1, rank))])
        return None, None, {"extra": {f"{name}:selectivity_eps": table}}
    raise KeyError(name)


def main(names):
    table = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            table = json.load(f)
    for n in names:
        key, eps, info = calibrate(n)
        if key is not None:
            table[key] = eps
        table.update(info.pop("extra", {}))
        print(n, key, repr(eps), info, file=sys.stderr)
        with open(OUT, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
            f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:] or ["rxs_histograms_2k", "self_clustered_262k", "rxs_unit_mixture_1m", "batch_store_2m",
                          "serve_store_4m", "hist_clustered_64k", "tracked_objects_262k"])
