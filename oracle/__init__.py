"""CPU oracle for the epsilon-similarity join -- TEST INFRASTRUCTURE, NOT THE PRODUCT.

Only tests/, the smoke check and the benchmark's CPU-baseline leg may import
this package. The CUDA library never calls it and shares no code with it.

`oracle.c` holds the definition (plain single-threaded FP64 nested loop, see its
header for the paper passages it follows); this module compiles it with
`-ffp-contract=off` (so the canonical sum is not contracted into FMAs on either
x86-64 or aarch64), loads it with ctypes and wraps numpy arrays.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]
LIBS = ["-lm"]

_lib = None


def build(src: str = _SRC, out: str = _LIB_PATH, extra=()) -> str:
    """Compile oracle.c into a shared library (gcc, no FMA contraction)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    cmd = ["gcc", *CFLAGS, *extra, "-o", out, src, *LIBS]
    subprocess.run(cmd, check=True)
    return out


def _needs_build(src: str, out: str) -> bool:
    return (not os.path.exists(out)) or os.path.getmtime(out) < os.path.getmtime(src)


def load(path: str | None = None):
    """Load (building if needed) the oracle library and declare its signatures."""
    global _lib
    if path is None:
        if _lib is not None:
            return _lib
        if _needs_build(_SRC, _LIB_PATH):
            build()
        path = _LIB_PATH
    lib = ctypes.CDLL(path)
    f32p = ctypes.POINTER(ctypes.c_float)
    f64p = ctypes.POINTER(ctypes.c_double)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_sqdist.restype = ctypes.c_double
    lib.oracle_sqdist.argtypes = [f32p, f32p, ctypes.c_int32]
    lib.oracle_join.restype = ctypes.c_int64
    lib.oracle_join.argtypes = [f32p, ctypes.c_int64, f32p, ctypes.c_int64, ctypes.c_int32,
                                ctypes.c_double, ctypes.c_int32, i64p, i64p, ctypes.c_int64]
    lib.oracle_dist_block.restype = None
    lib.oracle_dist_block.argtypes = [f32p, ctypes.c_int64, ctypes.c_int64, f32p, ctypes.c_int64,
                                      ctypes.c_int32, f64p]
    lib.oracle_normalize.restype = ctypes.c_int64
    lib.oracle_normalize.argtypes = [f32p, ctypes.c_int64, ctypes.c_int32, f32p]
    lib.oracle_cosine_join.restype = ctypes.c_int64
    lib.oracle_cosine_join.argtypes = [f32p, ctypes.c_int64, f32p, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_double, ctypes.c_int32, i64p, i64p, ctypes.c_int64]
    lib.oracle_topk.restype = ctypes.c_int32
    lib.oracle_topk.argtypes = [f32p, ctypes.c_int64, f32p, ctypes.c_int64, ctypes.c_int32,
                                ctypes.c_int32, i64p, f64p]
    u8p = ctypes.POINTER(ctypes.c_uint8)
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib.oracle_l1dist.restype = ctypes.c_double
    lib.oracle_l1dist.argtypes = [f32p, f32p, ctypes.c_int32]
    lib.oracle_chi2dist.restype = ctypes.c_double
    lib.oracle_chi2dist.argtypes = [f32p, f32p, ctypes.c_int32]
    lib.oracle_hist_join.restype = ctypes.c_int64
    lib.oracle_hist_join.argtypes = [f32p, ctypes.c_int64, f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_double, ctypes.c_int32, i64p, i64p, ctypes.c_int64]
    lib.oracle_hist_dist_block.restype = None
    lib.oracle_hist_dist_block.argtypes = [f32p, ctypes.c_int64, ctypes.c_int64, f32p, ctypes.c_int64,
                                           ctypes.c_int32, ctypes.c_int32, f64p]
    lib.oracle_color_hist.restype = ctypes.c_int64
    lib.oracle_color_hist.argtypes = [u8p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, i32p, ctypes.c_int64,
                                      ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, f32p]
    lib.oracle_hist_topk.restype = ctypes.c_int32
    lib.oracle_hist_topk.argtypes = [f32p, ctypes.c_int64, f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int32, i64p, f64p]
    lib.oracle_dot.restype = ctypes.c_double
    lib.oracle_dot.argtypes = [f32p, f32p, ctypes.c_int32]
    lib.oracle_ip_join.restype = ctypes.c_int64
    lib.oracle_ip_join.argtypes = [f32p, ctypes.c_int64, f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                   ctypes.c_int32, i64p, i64p, ctypes.c_int64]
    lib.oracle_components.restype = ctypes.c_int64
    lib.oracle_components.argtypes = [ctypes.c_int64, i64p, i64p, ctypes.c_int64, i64p]
    if path == _LIB_PATH:
        _lib = lib
    return lib


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


MODE_RXS, MODE_SELF_UPPER, MODE_SELF_FULL = 0, 1, 2
METRIC_L1, METRIC_CHI2 = 1, 2
DEDUP_ALL, DEDUP_FILTER_MATCH, DEDUP_MATCH_FILTER = 0, 1, 2


class Oracle:
    """Thin numpy wrapper over one loaded oracle library (the real one, or a test mutant)."""

    def __init__(self, lib=None):
        self.lib = lib if lib is not None else load()

    def sqdist(self, q, x) -> float:
        q, qp = _f32(q)
        x, xp = _f32(x)
        return float(self.lib.oracle_sqdist(qp, xp, int(q.shape[-1])))

    def dist_block(self, R, S, r0: int = 0, r1: int | None = None) -> np.ndarray:
        R, Rp = _f32(R)
        S, Sp = _f32(S)
        r1 = R.shape[0] if r1 is None else r1
        out = np.empty((r1 - r0, S.shape[0]), dtype=np.float64)
        self.lib.oracle_dist_block(Rp, r0, r1, Sp, S.shape[0], R.shape[1],
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return out

    def join(self, R, S=None, eps: float = 0.0, mode: int | None = None,
             cap: int | None = None) -> np.ndarray:
        """Row-index pairs (int64 [n, 2]) of the epsilon-join, in nested-loop order."""
        R, Rp = _f32(R)
        if mode is None:
            mode = MODE_RXS if S is not None else MODE_SELF_UPPER
        if S is None:
            S, Sp, nS = R, Rp, R.shape[0]
        else:
            S, Sp = _f32(S)
            nS = S.shape[0]
        d = R.shape[1]
        i64 = ctypes.POINTER(ctypes.c_int64)
        if cap is None:
            cap = 1 << 16
        while True:
            out_r = np.empty(cap, dtype=np.int64)
            out_s = np.empty(cap, dtype=np.int64)
            n = self.lib.oracle_join(Rp, R.shape[0], Sp, nS, d, float(eps), mode,
                                     out_r.ctypes.data_as(i64), out_s.ctypes.data_as(i64), cap)
            if n <= cap:
                return np.stack([out_r[:n], out_s[:n]], axis=1)
            cap = int(n)

    def normalize(self, X):
        """Unit-normalized copy (the cosine metric's rows); raises on a zero-norm row."""
        X, Xp = _f32(X)
        out = np.empty_like(X)
        bad = self.lib.oracle_normalize(Xp, X.shape[0], X.shape[1], out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        if bad:
            raise ValueError(f"{bad} rows have a zero norm")
        return out

    def cosine_join(self, Rn, Sn=None, c: float = 1.0, mode: int | None = None) -> np.ndarray:
        """Row-index pairs with canonical D(q^, x^) <= fl64(2 - 2c) on normalized rows."""
        Rn, Rp = _f32(Rn)
        if mode is None:
            mode = MODE_RXS if Sn is not None else MODE_SELF_UPPER
        if Sn is None:
            Sn, Sp, nS = Rn, Rp, Rn.shape[0]
        else:
            Sn, Sp = _f32(Sn)
            nS = Sn.shape[0]
        i64 = ctypes.POINTER(ctypes.c_int64)
        cap = 1 << 16
        while True:
            out_r = np.empty(cap, dtype=np.int64)
            out_s = np.empty(cap, dtype=np.int64)
            n = self.lib.oracle_cosine_join(Rp, Rn.shape[0], Sp, nS, Rn.shape[1], float(c), mode,
                                            out_r.ctypes.data_as(i64), out_s.ctypes.data_as(i64), cap)
            if n <= cap:
                return np.stack([out_r[:n], out_s[:n]], axis=1)
            cap = int(n)

    def hist_dist(self, q, x, metric: int) -> float:
        q, qp = _f32(q)
        x, xp = _f32(x)
        f = self.lib.oracle_l1dist if metric == METRIC_L1 else self.lib.oracle_chi2dist
        return float(f(qp, xp, int(q.shape[-1])))

    def hist_dist_block(self, R, S, metric: int, r0: int = 0, r1: int | None = None) -> np.ndarray:
        R, Rp = _f32(R)
        S, Sp = _f32(S)
        r1 = R.shape[0] if r1 is None else r1
        out = np.empty((r1 - r0, S.shape[0]), dtype=np.float64)
        self.lib.oracle_hist_dist_block(Rp, r0, r1, Sp, S.shape[0], R.shape[1], int(metric),
                                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return out

    def hist_join(self, R, S=None, eps: float = 0.0, metric: int = METRIC_L1, mode: int | None = None) -> np.ndarray:
        """Row-index pairs with canonical L1 (metric 1) or chi-square (metric 2) distance <= eps."""
        R, Rp = _f32(R)
        if mode is None:
            mode = MODE_RXS if S is not None else MODE_SELF_UPPER
        if S is None:
            S, Sp, nS = R, Rp, R.shape[0]
        else:
            S, Sp = _f32(S)
            nS = S.shape[0]
        i64 = ctypes.POINTER(ctypes.c_int64)
        cap = 1 << 16
        while True:
            out_r = np.empty(cap, dtype=np.int64)
            out_s = np.empty(cap, dtype=np.int64)
            n = self.lib.oracle_hist_join(Rp, R.shape[0], Sp, nS, R.shape[1], int(metric), float(eps), mode,
                                          out_r.ctypes.data_as(i64), out_s.ctypes.data_as(i64), cap)
            if n <= cap:
                return np.stack([out_r[:n], out_s[:n]], axis=1)
            cap = int(n)

    def dot(self, q, x) -> float:
        q, qp = _f32(q)
        x, xp = _f32(x)
        return float(self.lib.oracle_dot(qp, xp, int(q.shape[-1])))

    def ip_join(self, R, S=None, t: float = 0.0, mode: int | None = None) -> np.ndarray:
        """Row-index pairs with canonical inner product q.x >= t, in nested-loop order."""
        R, Rp = _f32(R)
        if mode is None:
            mode = MODE_RXS if S is not None else MODE_SELF_UPPER
        if S is None:
            S, Sp, nS = R, Rp, R.shape[0]
        else:
            S, Sp = _f32(S)
            nS = S.shape[0]
        i64 = ctypes.POINTER(ctypes.c_int64)
        cap = 1 << 16
        while True:
            out_r = np.empty(cap, dtype=np.int64)
            out_s = np.empty(cap, dtype=np.int64)
            n = self.lib.oracle_ip_join(Rp, R.shape[0], Sp, nS, R.shape[1], float(t), mode,
                                        out_r.ctypes.data_as(i64), out_s.ctypes.data_as(i64), cap)
            if n <= cap:
                return np.stack([out_r[:n], out_s[:n]], axis=1)
            cap = int(n)

    def hist_topk(self, Q, S, k: int, metric: int = METRIC_L1):
        """(idx int64 [nQ, k], dist float64 [nQ, k]) by (L1 or chi-square distance, store row); unused slots -1."""
        Q, Qp = _f32(Q)
        S, Sp = _f32(S)
        idx = np.empty((Q.shape[0], k), dtype=np.int64)
        dist = np.empty((Q.shape[0], k), dtype=np.float64)
        rc = self.lib.oracle_hist_topk(Qp, Q.shape[0], Sp, S.shape[0], Q.shape[1], int(metric), int(k),
                                       idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                       dist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        if rc != 0:
            raise MemoryError("oracle_hist_topk: allocation failed")
        return idx, dist

    def color_hist(self, frames, boxes, bins) -> np.ndarray:
        """Histograms [nb, br*bg*bb] of the boxes {frame, x0, y0, x1, y1} of frames [nF, H, W, 3] (uint8)."""
        frames = np.ascontiguousarray(frames, dtype=np.uint8)
        boxes = np.ascontiguousarray(boxes, dtype=np.int32).reshape(-1, 5)
        br, bg, bb = (int(b) for b in bins)
        out = np.empty((boxes.shape[0], br * bg * bb), dtype=np.float32)
        rc = self.lib.oracle_color_hist(frames.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), frames.shape[0],
                                        frames.shape[1], frames.shape[2],
                                        boxes.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), boxes.shape[0],
                                        br, bg, bb, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        if rc < 0:
            raise MemoryError("oracle_color_hist: allocation failed")
        if rc > 0:
            raise ValueError(f"box {rc - 1} is invalid")
        return out

    def components(self, n: int, pairs) -> tuple[np.ndarray, int]:
        """(label int64 [n], number of components): label = smallest row index of the component."""
        pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int64).reshape(-1, 2))
        a = np.ascontiguousarray(pairs[:, 0])
        b = np.ascontiguousarray(pairs[:, 1])
        label = np.empty(n, dtype=np.int64)
        i64 = ctypes.POINTER(ctypes.c_int64)
        c = self.lib.oracle_components(int(n), a.ctypes.data_as(i64), b.ctypes.data_as(i64), a.shape[0],
                                       label.ctypes.data_as(i64))
        if c < 0:
            raise ValueError("an edge names a row outside [0, n)")
        return label, int(c)

    def dedup(self, X, eps: float, labels=None, target: int = 0, plan: int = DEDUP_ALL):
        """q4 (Sec. 6.2, Sec. 7.4.3): (component label per row, number of distinct objects).

        DEDUP_ALL: components of the epsilon self-join of every row.
        DEDUP_FILTER_MATCH: keep the rows whose label is `target`, join them, count their
          components; the other rows get label -1.
        DEDUP_MATCH_FILTER: join every row, then count the components holding at least
          one row whose label is `target`.
        """
        X = np.ascontiguousarray(X, dtype=np.float32)
        n = X.shape[0]
        if plan == DEDUP_FILTER_MATCH:
            keep = np.flatnonzero(np.asarray(labels) == target)
            pairs = keep[self.join(X[keep], None, eps, MODE_SELF_UPPER)] if keep.size else np.empty((0, 2), np.int64)
            lab, _ = self.components(n, pairs)
            out = np.full(n, -1, dtype=np.int64)
            out[keep] = lab[keep]
            return out, int(np.unique(lab[keep]).size)
        lab, c = self.components(n, self.join(X, None, eps, MODE_SELF_UPPER))
        if plan == DEDUP_ALL:
            return lab, c
        hit = np.asarray(labels) == target
        return lab, int(np.unique(lab[hit]).size)

    def topk(self, Q, S, k: int):
        """(idx int64 [nQ, k], d2 float64 [nQ, k]); unused slots are -1."""
        Q, Qp = _f32(Q)
        S, Sp = _f32(S)
        idx = np.empty((Q.shape[0], k), dtype=np.int64)
        d2 = np.empty((Q.shape[0], k), dtype=np.float64)
        rc = self.lib.oracle_topk(Qp, Q.shape[0], Sp, S.shape[0], Q.shape[1], int(k),
                                  idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  d2.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        if rc != 0:
            raise MemoryError("oracle_topk: allocation failed")
        return idx, d2


_default = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle()
    return _default


if __name__ == "__main__":
    build()
    print("built", _LIB_PATH, file=sys.stderr)
