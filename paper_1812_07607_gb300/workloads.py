"""Seeded synthetic patch-feature workloads for the epsilon-similarity join.

This module only *draws inputs*: feature matrices, patch ids and request mixes.
It contains none of the join's arithmetic (no distances, norms or thresholds),
so both the CUDA path (tests, bench) and the CPU oracle's tests can take their
inputs from it without sharing any of the method.

The paper's datasets (PC, TrafficCam, Football; Sec. 6.1) are not available,
so these generators stand in for them. The feature the paper joins on is a
colour histogram (Sec. 4.1, "Transformers"): a non-negative vector that sums
to one. Repeated objects across video frames (q4, Sec. 6.2) are mimicked by
jittered copies of shared centroids.

Every generator is a pure function of its arguments and a numpy PCG64 seed.
All draws are made in float64 and cast to float32 once; the float32 values are
the ground truth that every implementation consumes.
"""

from __future__ import annotations

import json
import os
from dataclasses import dataclass

import numpy as np

SEED_BASE = 1812076070

_EPS_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workload_eps.json")


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def dirichlet_histograms(g: np.random.Generator, n: int, d: int, alpha: float = 0.5,
                         chunk: int = 65536) -> np.ndarray:
    """n colour-histogram rows drawn i.i.d. from Dirichlet(alpha * 1_d)."""
    out = np.empty((n, d), dtype=np.float32)
    a = np.full(d, alpha, dtype=np.float64)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        out[r0:r1] = g.dirichlet(a, size=r1 - r0).astype(np.float32)
    return out


def clustered_histograms(g: np.random.Generator, n: int, d: int, n_centroids: int,
                         sigma: float, alpha: float = 0.5, chunk: int = 65536):
    """Histograms of repeated objects: Dirichlet centroids plus Gaussian jitter.

    Each row picks a centroid uniformly, adds N(0, sigma^2) per bin, clips at
    zero and renormalises to sum one (a row that clips to all-zero keeps its
    centroid). Returns (features float32 [n, d], centroid index int64 [n]).
    """
    cents = g.dirichlet(np.full(d, alpha, dtype=np.float64), size=n_centroids)
    assign = g.integers(0, n_centroids, size=n, dtype=np.int64)
    out = np.empty((n, d), dtype=np.float32)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        c = cents[assign[r0:r1]]
        x = c + g.normal(0.0, sigma, size=(r1 - r0, d))
        np.clip(x, 0.0, None, out=x)
        s = x.sum(axis=1, keepdims=True)
        bad = (s[:, 0] <= 0.0)
        if bad.any():
            x[bad] = c[bad]
            s[bad] = 1.0
        out[r0:r1] = (x / s).astype(np.float32)
    return out, assign


def unit_mixture(g: np.random.Generator, n: int, d: int, n_centroids: int, sigma: float,
                 chunk: int = 65536, centroids: np.ndarray | None = None):
    """Unit-norm embeddings from a Gaussian mixture on the sphere.

    Centroids are uniform on S^{d-1} (normalised standard normals) unless given;
    a row is its centroid plus N(0, sigma^2 I), renormalised to unit length.
    Returns (features float32 [n, d], centroids float64 [C, d]).
    """
    if centroids is None:
        c = g.normal(size=(n_centroids, d))
        centroids = c / np.linalg.norm(c, axis=1, keepdims=True)
    assign = g.integers(0, centroids.shape[0], size=n, dtype=np.int64)
    out = np.empty((n, d), dtype=np.float32)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        x = centroids[assign[r0:r1]] + g.normal(0.0, sigma, size=(r1 - r0, d))
        x /= np.linalg.norm(x, axis=1, keepdims=True)
        out[r0:r1] = x.astype(np.float32)
    return out, centroids


def patch_ids(g: np.random.Generator, n: int) -> np.ndarray:
    """Opaque int64 patch ids: a random permutation of a sparse id space."""
    base = g.permutation(n).astype(np.int64)
    return base * 7919 + 1_000_003


def eps_for_selectivity(table, sel: float) -> float:
    """eps for a target selectivity from a stored (selectivity, eps) table (log-linear interpolation)."""
    t = np.asarray(table, dtype=np.float64)
    return float(np.interp(np.log(sel), np.log(t[:, 0]), t[:, 1]))


def eps_table() -> dict:
    """Calibrated epsilon per named workload (written by the oracle's calibration)."""
    with open(_EPS_FILE) as f:
        return json.load(f)


# --------------------------------------------------------------------------------------
# Named workloads. Each returns plain numpy arrays; nothing is placed on a device here.
# --------------------------------------------------------------------------------------

@dataclass
class JoinWorkload:
    name: str
    R: np.ndarray            # float32 [nR, d]
    S: np.ndarray | None     # float32 [nS, d]; None for a self-join of R
    r_ids: np.ndarray        # int64 [nR]
    s_ids: np.ndarray | None
    eps: float
    groups: np.ndarray | None = None   # int64 [nR]: the object (centroid) each row is a view of

    @property
    def d(self) -> int:
        return int(self.R.shape[1])

    @property
    def pairs(self) -> int:
        """Pairs the join evaluates: |R||S|, or N(N-1)/2 for an (upper) self-join."""
        n = self.R.shape[0]
        if self.S is None:
            return n * (n - 1) // 2
        return n * self.S.shape[0]


def rxs_histograms_2k(seed: int = SEED_BASE + 0, n: int = 2000, d: int = 64,
                      eps: float | None = None) -> JoinWorkload:
    """R x S join of two 2,000-patch sets of d=64 Dirichlet(0.5) colour histograms."""
    g = rng(seed)
    R = dirichlet_histograms(g, n, d)
    S = dirichlet_histograms(g, n, d)
    rid = patch_ids(g, n)
    sid = patch_ids(g, n) + 10**12
    if eps is None:
        eps = eps_table().get(f"rxs_histograms_2k:{seed}:{n}:{d}")
    return JoinWorkload("rxs_histograms_2k", R, S, rid, sid, eps)


def self_clustered_262k(seed: int = SEED_BASE + 1, n: int = 262144, d: int = 128,
                        n_centroids: int = 8192, sigma: float = 0.01,
                        eps: float | None = None) -> JoinWorkload:
    """Self-join of 262,144 d=128 histograms: 8,192 Dirichlet centroids + N(0, 0.01^2) jitter."""
    g = rng(seed)
    X, groups = clustered_histograms(g, n, d, n_centroids, sigma)
    ids = patch_ids(g, n)
    if eps is None:
        eps = eps_table().get(f"self_clustered_262k:{seed}:{n}:{d}:{n_centroids}")
    return JoinWorkload("self_clustered_262k", X, None, ids, None, eps, groups)


def hist_clustered_64k(seed: int = SEED_BASE + 6, n: int = 65536, d: int = 128, n_centroids: int = 2048,
                       sigma: float = 0.01):
    """Self-join store of the histogram metrics (L1, chi-square): 65,536 d=128 clustered
    histograms (2,048 Dirichlet(0.5) centroids + N(0, 0.01^2) jitter, clipped, renormalised;
    clipping leaves exact zero bins). Returns (features, {metric: eps}) with eps from the
    oracle-calibrated table (about 20 other rows within eps per row)."""
    g = rng(seed)
    X, _ = clustered_histograms(g, n, d, n_centroids, sigma)
    tab = eps_table()
    return X, {m: tab.get(f"hist_clustered_64k:{m}:{seed}") for m in ("l1", "chi2")}


def tracked_objects_262k(seed: int = SEED_BASE + 7, n: int = 262144, d: int = 128, n_objects: int = 256,
                         sigma: float = 0.003, eps: float | None = None) -> JoinWorkload:
    """Self-join store of the pruned join: 262,144 d=128 patch histograms of 256 tracked objects
    (about 1,024 views each, as a pedestrian or vehicle seen over many frames; q4), each view its
    object's Dirichlet(0.5) histogram plus N(0, 0.003^2) jitter, clipped and renormalised.
    eps from the oracle-calibrated table: a mean of 100 other rows within eps per row."""
    g = rng(seed)
    X, groups = clustered_histograms(g, n, d, n_objects, sigma)
    ids = patch_ids(g, n)
    if eps is None:
        eps = eps_table().get(f"tracked_objects_262k:{seed}:{n}:{d}:{n_objects}")
    return JoinWorkload("tracked_objects_262k", X, None, ids, None, eps, groups)


def clustered_queries(n: int, seed_q: int, store_seed: int, d: int, n_centroids: int, sigma: float,
                      alpha: float = 0.5) -> np.ndarray:
    """Fresh query patches for a clustered store: new jitters of the store's own centroids.

    The store generator draws its centroids first from rng(store_seed), so they are
    re-drawn here the same way; the jitter follows clustered_histograms.
    """
    cents = rng(store_seed).dirichlet(np.full(d, alpha, dtype=np.float64), size=n_centroids)
    g = rng(seed_q)
    out = np.empty((n, d), dtype=np.float32)
    chunk = 65536
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        c = cents[g.integers(0, n_centroids, size=r1 - r0)]
        x = np.clip(c + g.normal(0.0, sigma, size=(r1 - r0, d)), 0.0, None)
        s = x.sum(axis=1, keepdims=True)
        bad = s[:, 0] <= 0.0
        x[bad] = c[bad]
        s[bad] = 1.0
        out[r0:r1] = (x / s).astype(np.float32)
    return out


def self_clustered_queries(n: int, seed_q: int, seed: int = SEED_BASE + 1, d: int = 128,
                           n_centroids: int = 8192, sigma: float = 0.01) -> np.ndarray:
    """Fresh query patches for the 262,144-patch store: new jitters of the store's own centroids."""
    return clustered_queries(n, seed_q, seed, d, n_centroids, sigma)


@dataclass
class StoreWorkload:
    name: str
    X: np.ndarray            # float32 [n, d]
    ids: np.ndarray          # int64 [n]
    seed: int
    n_centroids: int
    sigma: float

    @property
    def d(self) -> int:
        return int(self.X.shape[1])

    def queries(self, n: int, seed_q: int) -> np.ndarray:
        return clustered_queries(n, seed_q, self.seed, self.d, self.n_centroids, self.sigma)

    def eps_table(self):
        """(selectivity, eps) pairs calibrated by the oracle on this store."""
        return eps_table()[f"{self.name}:selectivity_eps"]


def batch_store_2m(seed: int = SEED_BASE + 3, n: int = 2097152, d: int = 128, n_centroids: int = 65536,
                   sigma: float = 0.01) -> StoreWorkload:
    """Shared store of the batched-requests workload: 2,097,152 d=128 clustered histograms."""
    X, _ = clustered_histograms(rng(seed), n, d, n_centroids, sigma)
    return StoreWorkload("batch_store_2m", X, patch_ids(rng(seed + 1000), n), seed, n_centroids, sigma)


def serve_store_4m(seed: int = SEED_BASE + 4, n: int = 4194304, d: int = 256, n_centroids: int = 131072,
                   sigma: float = 0.01) -> StoreWorkload:
    """Device-resident store of the serving workload: 4,194,304 d=256 clustered histograms."""
    X, _ = clustered_histograms(rng(seed), n, d, n_centroids, sigma)
    return StoreWorkload("serve_store_4m", X, patch_ids(rng(seed + 1000), n), seed, n_centroids, sigma)


def rxs_unit_mixture_1m(seed: int = SEED_BASE + 2, n: int = 1048576, d: int = 512,
                        n_centroids: int = 4096, sigma: float = 0.02,
                        eps: float | None = None) -> JoinWorkload:
    """R x S join of unit-norm d=512 embeddings drawn from one 4,096-component mixture."""
    g = rng(seed)
    R, cents = unit_mixture(g, n, d, n_centroids, sigma)
    S, _ = unit_mixture(g, n, d, n_centroids, sigma, centroids=cents)
    rid = patch_ids(g, n)
    sid = patch_ids(g, n) + 10**12
    if eps is None:
        eps = eps_table().get(f"rxs_unit_mixture_1m:{seed}:{n}:{d}:{n_centroids}")
    return JoinWorkload("rxs_unit_mixture_1m", R, S, rid, sid, eps)


# --------------------------------------------------------------------------------------
# Small adversarial / closed-form inputs used by the tests of both sides.
# --------------------------------------------------------------------------------------

def grid_points(g: np.random.Generator, n: int, d: int, levels: int = 8, shift: int = 3,
                dup_frac: float = 0.0) -> np.ndarray:
    """Integer grid values scaled by 2^-shift: exact in FP32, BF16 and FP64.

    With dup_frac > 0 a fraction of rows are copies of earlier rows (exact duplicates).
    """
    X = g.integers(0, levels, size=(n, d)).astype(np.float64) * (2.0 ** -shift)
    if dup_frac > 0 and n > 1:
        k = max(1, int(n * dup_frac))
        dst = g.choice(np.arange(1, n), size=min(k, n - 1), replace=False)
        for t in dst:
            X[t] = X[g.integers(0, t)]
    return X.astype(np.float32)


def one_hot_rows(g: np.random.Generator, n: int, d: int) -> np.ndarray:
    """Rows with a single 1 in a random bin: distinct rows are sqrt(2) apart."""
    X = np.zeros((n, d), dtype=np.float32)
    X[np.arange(n), g.integers(0, d, size=n)] = 1.0
    return X


def mixed_magnitude_rows(g: np.random.Generator, n: int, d: int) -> np.ndarray:
    """Rows mixing widely different exponents, to exercise rounding in the distance sum."""
    mant = g.uniform(-1.0, 1.0, size=(n, d))
    expo = g.integers(-30, 8, size=(n, d))
    return (mant * np.exp2(expo)).astype(np.float32)


def request_mix(g: np.random.Generator, n_requests: int, mu: float, sigma: float,
                q_max: int, topk_frac: float, ks=(10,), sel_lo: float = 5e-4,
                sel_hi: float = 5e-3):
    """A batch of join / top-k requests with lognormal query-set sizes.

    Returns a list of dicts {kind: 'eps'|'topk', nq, k, selectivity}. Sizes are
    round(lognormal(mu, sigma)) clipped to [1, q_max]; the kind is top-k with
    probability topk_frac (k uniform over ks), else an epsilon-join whose target
    selectivity is uniform in [sel_lo, sel_hi].
    """
    sizes = np.clip(np.rint(g.lognormal(mu, sigma, size=n_requests)), 1, q_max).astype(np.int64)
    kinds = g.uniform(size=n_requests) < topk_frac
    kk = g.choice(np.asarray(ks, dtype=np.int64), size=n_requests)
    sel = g.uniform(sel_lo, sel_hi, size=n_requests)
    out = []
    for i in range(n_requests):
        if kinds[i]:
            out.append({"kind": "topk", "nq": int(sizes[i]), "k": int(kk[i]), "selectivity": None})
        else:
            out.append({"kind": "eps", "nq": int(sizes[i]), "k": 0, "selectivity": float(sel[i])})
    return out


def sample_rows(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct row indices of [0, n), ascending, drawn with a seeded permutation."""
    return np.sort(rng(seed).choice(n, size=min(k, n), replace=False)).astype(np.int64)


# Row sample of the 1,048,576 x 1,048,576 d=512 join whose exact pair set is stored as a digest.
UNIT_MIXTURE_SAMPLE_SEED = SEED_BASE + 103
UNIT_MIXTURE_SAMPLE_ROWS = 16384


# ---------------------------------------------------------------------------------------------
# detector output for q4 and raw frames for the colour-histogram transformer
# ---------------------------------------------------------------------------------------------

def object_labels(g: np.random.Generator, groups: np.ndarray, n_groups: int,
                  classes=(0.45, 0.45, 0.10), flip: float = 0.08) -> np.ndarray:
    """Detector labels of patches (q4): each object has a class (0 person, 1 vehicle, 2 other);
    each patch shows its object's class, except with probability `flip`, where the detector
    reports a uniformly drawn class instead. int32 [n]."""
    cls = g.choice(len(classes), size=n_groups, p=np.asarray(classes, dtype=np.float64))
    lab = cls[groups].astype(np.int32)
    f = g.random(len(groups)) < flip
    lab[f] = g.integers(0, len(classes), size=int(f.sum()), dtype=np.int32)
    return lab


def traffic_frames(g: np.random.Generator, n_frames: int, H: int = 1080, W: int = 1920,
                   block: int = 24, noise: int = 6) -> np.ndarray:
    """8-bit RGB frames [n, H, W, 3] (interleaved, row-major): piecewise-constant colour blocks
    (road, vehicles, sky stand-ins) plus uniform integer noise in [-noise, noise], clipped."""
    out = np.empty((n_frames, H, W, 3), dtype=np.uint8)
    bh, bw = -(-H // block), -(-W // block)
    for f in range(n_frames):
        base = g.integers(0, 256, size=(bh, bw, 3), dtype=np.int16)
        img = np.repeat(np.repeat(base, block, axis=0), block, axis=1)[:H, :W]
        img = img + g.integers(-noise, noise + 1, size=(H, W, 3), dtype=np.int16)
        np.clip(img, 0, 255, out=img)
        out[f] = img.astype(np.uint8)
    return out


DETECTOR_BOX_SIDES = np.array([16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512], dtype=np.int64)
DETECTOR_BOX_WEIGHTS = np.array([4, 6, 8, 9, 9, 8, 6, 4, 3, 2, 1], dtype=np.float64)


def detector_boxes(g: np.random.Generator, n_frames: int, H: int, W: int, per_frame: int) -> np.ndarray:
    """Object-detector boxes {frame, x0, y0, x1, y1} (int32 [n_frames * per_frame, 5], half-open):
    sides from a discrete log-spaced mix (16 to 512 pixels, small boxes most common), each
    jittered by up to a quarter, aspect 1:2 to 2:1, placed uniformly inside the frame."""
    n = n_frames * per_frame
    p = DETECTOR_BOX_WEIGHTS / DETECTOR_BOX_WEIGHTS.sum()
    side = g.choice(DETECTOR_BOX_SIDES, size=n, p=p)
    w = side + g.integers(-(side // 4), side // 4 + 1)
    h = (w * g.integers(2, 9, size=n)) // 4
    w = np.clip(w, 1, W)
    h = np.clip(h, 1, H)
    x0 = g.integers(0, W - w + 1)
    y0 = g.integers(0, H - h + 1)
    f = np.repeat(np.arange(n_frames, dtype=np.int64), per_frame)
    return np.stack([f, x0, y0, x0 + w, y0 + h], axis=1).astype(np.int32)


@dataclass
class FrameWorkload:
    name: str
    frames: np.ndarray       # uint8 [n_frames, H, W, 3]
    boxes: np.ndarray        # int32 [n_boxes, 5]
    bins: tuple              # (br, bg, bb)

    @property
    def pixels(self) -> int:
        b = self.boxes.astype(np.int64)
        return int(((b[:, 3] - b[:, 1]) * (b[:, 4] - b[:, 2])).sum())


def traffic_boxes_1080p(seed: int = SEED_BASE + 5, n_frames: int = 64, per_frame: int = 64,
                        bins=(8, 4, 4)) -> FrameWorkload:
    """64 1080p frames with 64 detector boxes each, histograms of (8, 4, 4) = 128 bins."""
    g = rng(seed)
    frames = traffic_frames(g, n_frames)
    boxes = detector_boxes(g, n_frames, frames.shape[1], frames.shape[2], per_frame)
    return FrameWorkload("traffic_boxes_1080p", frames, boxes, tuple(bins))
