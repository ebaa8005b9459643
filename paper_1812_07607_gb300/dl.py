"""Thin ctypes binding of the C ABI declared in include/dl.h.

Argument marshalling only: every step of the join runs in the library's CUDA
kernels. PyTorch supplies device memory and streams. There is no CPU
fallback: if the library is missing or no GB300 is usable, calls raise.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdlsimjoin.so")
CHECKED_LIB_PATH = os.path.join(HERE, "libdlsimjoin_checked.so")   # the bounds-checked build (build(checked=True))

# dl_status
DL_OK, DL_EINVAL, DL_ENOMEM, DL_EOVERFLOW, DL_EAGAIN, DL_ETIMEOUT, DL_ECUDA, DL_ECANCELED, \
    DL_ENOMEM_ADMIT, DL_EFAILED, DL_EUNSUPPORTED = range(11)
STATUS_NAMES = {0: "DL_OK", 1: "DL_EINVAL", 2: "DL_ENOMEM", 3: "DL_EOVERFLOW", 4: "DL_EAGAIN",
                5: "DL_ETIMEOUT", 6: "DL_ECUDA", 7: "DL_ECANCELED", 8: "DL_ENOMEM_ADMIT",
                9: "DL_EFAILED", 10: "DL_EUNSUPPORTED"}
DL_METRIC_L2, DL_METRIC_COSINE, DL_METRIC_L1, DL_METRIC_CHI2, DL_METRIC_IP = 0, 1, 2, 3, 4
METRICS = {"l2": DL_METRIC_L2, "cosine": DL_METRIC_COSINE, "l1": DL_METRIC_L1, "chi2": DL_METRIC_CHI2, "ip": DL_METRIC_IP}
DL_DEDUP_ALL, DL_DEDUP_FILTER_MATCH, DL_DEDUP_MATCH_FILTER = 0, 1, 2
DEDUP_PLANS = {"all": DL_DEDUP_ALL, "filter_match": DL_DEDUP_FILTER_MATCH, "match_filter": DL_DEDUP_MATCH_FILTER}
DL_PREC_AUTO, DL_PREC_BF16, DL_PREC_FP8E4M3, DL_PREC_FP32, DL_PREC_FP32_PLAIN = range(5)
PRECISIONS = {"auto": 0, "bf16": 1, "fp8": 2, "fp32": 3, "fp32_plain": 4}
DL_MEM_HOST, DL_MEM_DEVICE = 0, 1
DL_SELF_UPPER, DL_SELF_FULL = 0, 1

# Every function include/dl.h declares (checked by the CPU test suite).
EXPORTS = [
    "dl_join_opts_default", "dl_store_create", "dl_store_destroy", "dl_store_shape",
    "dl_sim_join", "dl_topk_join", "dl_result_count", "dl_result_pairs", "dl_result_topk",
    "dl_result_stats", "dl_result_free", "dl_last_error", "dl_version", "dl_kernel_launches",
    "dl_sim_join_noalloc", "dl_batch_join", "dl_result_request_pairs", "dl_result_request_topk",
    "dl_server_create", "dl_submit", "dl_poll", "dl_cancel", "dl_server_get_stats", "dl_server_destroy",
    "dl_debug_scores", "dl_store_normalize", "dl_color_hist", "dl_components", "dl_dedup", "dl_store_cluster",
    "dl_debug_set_wait_budget", "dl_debug_check_word", "dl_debug_check_selftest",
]


class DLError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class dl_join_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("self_mode", ctypes.c_int32),
                ("out_capacity", ctypes.c_int64), ("cuda_stream", ctypes.c_void_p),
                ("tile_n", ctypes.c_int32), ("timing", ctypes.c_int32), ("prune", ctypes.c_int32),
                ("cta_pair", ctypes.c_int32), ("epilogue_warps", ctypes.c_int32)]


class dl_join_stats(ctypes.Structure):
    _fields_ = [("pairs_evaluated", ctypes.c_int64), ("pairs_out", ctypes.c_int64),
                ("band_pairs", ctypes.c_int64), ("fp64_pairs", ctypes.c_int64),
                ("reruns", ctypes.c_int64), ("precision", ctypes.c_int32), ("tile_n", ctypes.c_int32),
                ("ms_main", ctypes.c_float), ("ms_recheck", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("kernels_launched", ctypes.c_int32), ("tile_pairs", ctypes.c_int64),
                ("tile_pairs_kept", ctypes.c_int64), ("cta_pair", ctypes.c_int32),
                ("grid_ctas", ctypes.c_int32), ("epilogue_warps", ctypes.c_int32)]


class dl_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("k", ctypes.c_int32), ("eps", ctypes.c_double),
                ("q_begin", ctypes.c_int64), ("nq", ctypes.c_int64)]


DL_REQ_EPS, DL_REQ_TOPK = 0, 1


class dl_server_stats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("failed", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("in_flight_batches", ctypes.c_int32),
                ("admission_waits", ctypes.c_int64), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("mean_ms", ctypes.c_double), ("mean_batch_requests", ctypes.c_double)]

_lib = None


def lib_path() -> str:
    return LIB_PATH


def load(path: str | None = None):
    """Load the C-ABI library (raises if it has not been built) and make it the one every call of
    this binding uses: the in-tree build, or the library at `path` (e.g. the bounds-checked build)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run paper_1812_07607_gb300.build)")
    L = ctypes.CDLL(path)
    vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    pp = ctypes.POINTER(ctypes.c_void_p)
    L.dl_join_opts_default.argtypes = [ctypes.POINTER(dl_join_opts)]
    L.dl_join_opts_default.restype = None
    L.dl_store_create.argtypes = [pp, vp, vp, i64, i32, i32, vp]
    L.dl_store_destroy.argtypes = [vp]
    L.dl_store_shape.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i32)]
    L.dl_store_normalize.argtypes = [vp, pp, vp]
    L.dl_store_normalize.restype = ctypes.c_int
    L.dl_sim_join.argtypes = [vp, vp, i32, f64, ctypes.POINTER(dl_join_opts), pp]
    L.dl_topk_join.argtypes = [vp, vp, i32, i32, ctypes.POINTER(dl_join_opts), pp]
    L.dl_result_count.argtypes = [vp, ctypes.POINTER(i64)]
    L.dl_result_pairs.argtypes = [vp, i32, pp, pp, ctypes.POINTER(i64)]
    L.dl_result_topk.argtypes = [vp, i32, pp, pp, ctypes.POINTER(i32), ctypes.POINTER(i64)]
    L.dl_result_stats.argtypes = [vp, ctypes.POINTER(dl_join_stats)]
    L.dl_result_free.argtypes = [vp]
    L.dl_sim_join_noalloc.argtypes = [vp, vp, i64, vp, vp, i64, i32, f64, i32, vp, vp, i64,
                                      ctypes.POINTER(i64), vp]
    L.dl_sim_join_noalloc.restype = ctypes.c_int
    L.dl_batch_join.argtypes = [vp, vp, vp, i64, i32, i32, ctypes.POINTER(dl_request), i32,
                                ctypes.POINTER(dl_join_opts), pp]
    L.dl_batch_join.restype = ctypes.c_int
    L.dl_result_request_pairs.argtypes = [vp, i32, i32, pp, pp, ctypes.POINTER(i64)]
    L.dl_result_request_pairs.restype = ctypes.c_int
    L.dl_result_request_topk.argtypes = [vp, i32, i32, pp, pp, ctypes.POINTER(i32), ctypes.POINTER(i64)]
    L.dl_result_request_topk.restype = ctypes.c_int
    L.dl_server_create.argtypes = [pp, vp, i64, i32, i64, ctypes.POINTER(dl_join_opts)]
    L.dl_submit.argtypes = [vp, vp, vp, i64, i32, f64, i32, ctypes.POINTER(ctypes.c_uint64)]
    L.dl_poll.argtypes = [vp, ctypes.c_uint64, i64, pp]
    L.dl_cancel.argtypes = [vp, ctypes.c_uint64]
    L.dl_server_get_stats.argtypes = [vp, ctypes.POINTER(dl_server_stats)]
    L.dl_server_destroy.argtypes = [vp]
    for name in ("dl_server_create", "dl_submit", "dl_poll", "dl_cancel", "dl_server_get_stats", "dl_server_destroy"):
        getattr(L, name).restype = ctypes.c_int
    L.dl_store_cluster.argtypes = [vp, i32, i32, pp, vp]
    L.dl_store_cluster.restype = ctypes.c_int
    L.dl_color_hist.argtypes = [vp, i64, i32, i32, vp, i64, i32, i32, i32, vp, ctypes.POINTER(ctypes.c_float), vp]
    L.dl_color_hist.restype = ctypes.c_int
    L.dl_components.argtypes = [i64, vp, vp, i64, vp, ctypes.POINTER(i64), vp]
    L.dl_components.restype = ctypes.c_int
    L.dl_dedup.argtypes = [vp, i32, f64, vp, i32, i32, ctypes.POINTER(dl_join_opts), vp, ctypes.POINTER(i64)]
    L.dl_dedup.restype = ctypes.c_int
    L.dl_debug_scores.argtypes = [vp, vp, i32, vp, vp, vp]
    L.dl_debug_scores.restype = ctypes.c_int
    L.dl_debug_set_wait_budget.argtypes = [i64]
    L.dl_debug_set_wait_budget.restype = ctypes.c_int
    L.dl_debug_check_word.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
    L.dl_debug_check_word.restype = ctypes.c_int
    L.dl_debug_check_selftest.argtypes = [i64]
    L.dl_debug_check_selftest.restype = ctypes.c_int
    L.dl_last_error.restype = ctypes.c_char_p
    L.dl_version.restype = ctypes.c_char_p
    L.dl_kernel_launches.restype = i64
    for name in ("dl_store_create", "dl_store_destroy", "dl_store_shape", "dl_sim_join", "dl_topk_join",
                 "dl_result_count", "dl_result_pairs", "dl_result_topk", "dl_result_stats",
                 "dl_result_free"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int, what: str):
    if rc != DL_OK:
        msg = load().dl_last_error().decode(errors="replace")
        raise DLError(rc, f"{what}: {msg}")


def last_error() -> str:
    return load().dl_last_error().decode(errors="replace")


def kernel_launches() -> int:
    return int(load().dl_kernel_launches())


def version() -> str:
    return load().dl_version().decode()


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class _DevView:
    """Expose a library-owned device buffer to torch through __cuda_array_interface__."""

    def __init__(self, ptr: int, n: int, typestr: str, owner):
        self._owner = owner
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                         "version": 2, "strides": None}


class Store:
    """A device-resident patch store (ids + float32 features), see dl_store_create."""

    def __init__(self, ids, feats, stream=None):
        L = load()
        h = ctypes.c_void_p()
        if hasattr(feats, "data_ptr"):   # torch tensor: device, or (pinned) host memory
            import torch
            feats = feats.contiguous().to(torch.float32)
            ids = ids.contiguous().to(device=feats.device, dtype=torch.int64)
            n, d = feats.shape
            where = DL_MEM_DEVICE if feats.is_cuda else DL_MEM_HOST
            st = _stream_handle(stream)
            rc = L.dl_store_create(ctypes.byref(h), ids.data_ptr(), feats.data_ptr(), n, d, where, st)
        else:
            feats = np.ascontiguousarray(feats, dtype=np.float32)
            ids = np.ascontiguousarray(ids, dtype=np.int64)
            n, d = feats.shape
            st = 0 if stream is None else _stream_handle(stream)
            rc = L.dl_store_create(ctypes.byref(h), ids.ctypes.data, feats.ctypes.data, n, d, DL_MEM_HOST, st)
        _check(rc, "dl_store_create")
        self._h = h
        self._lib = L   # the library that owns the store releases it
        self.n, self.d = int(n), int(d)

    @property
    def handle(self):
        return self._h

    def normalized(self, stream=None) -> "Store":
        """dl_store_normalize: a new store of the unit-normalized rows (for metric="cosine")."""
        h = ctypes.c_void_p()
        _check(self._lib.dl_store_normalize(self._h, ctypes.byref(h), _stream_handle(stream)), "dl_store_normalize")
        out = Store.__new__(Store)
        out._h = h
        out._lib = self._lib
        out.n, out.d = self.n, self.d
        return out

    def clustered(self, n_clusters: int, iters: int = 4, stream=None) -> "Store":
        """dl_store_cluster: the same rows in a k-means-grouped order (for sim_join(prune=True))."""
        h = ctypes.c_void_p()
        _check(self._lib.dl_store_cluster(self._h, int(n_clusters), int(iters), ctypes.byref(h),
                                          _stream_handle(stream)), "dl_store_cluster")
        out = Store.__new__(Store)
        out._h = h
        out._lib = self._lib
        out.n, out.d = self.n, self.d
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            (getattr(self, "_lib", None) or load()).dl_store_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _is_torch_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and bool(getattr(x, "is_cuda"))


class Result:
    """A join result owned by the library (dl_result)."""

    def __init__(self, h):
        self._h = h

    def count(self) -> int:
        n = ctypes.c_int64()
        _check(load().dl_result_count(self._h, ctypes.byref(n)), "dl_result_count")
        return int(n.value)

    def stats(self) -> dict:
        st = dl_join_stats()
        _check(load().dl_result_stats(self._h, ctypes.byref(st)), "dl_result_stats")
        return {f: getattr(st, f) for f, _ in dl_join_stats._fields_}

    def pairs_host(self, copy: bool = True):
        """(r_ids, s_ids) as int64 numpy arrays.

        copy=False returns views of the result's pinned host buffer: no host-side copy, valid
        until free() (the views do not keep the result alive).
        """
        a, b, n = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_int64()
        _check(load().dl_result_pairs(self._h, DL_MEM_HOST, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)),
               "dl_result_pairs")
        n = int(n.value)
        if n == 0:
            return np.empty(0, np.int64), np.empty(0, np.int64)
        ra = np.ctypeslib.as_array(ctypes.cast(a, ctypes.POINTER(ctypes.c_int64)), shape=(n,))
        sa = np.ctypeslib.as_array(ctypes.cast(b, ctypes.POINTER(ctypes.c_int64)), shape=(n,))
        return (ra.copy(), sa.copy()) if copy else (ra, sa)

    def pairs_device(self):
        """(r_ids, s_ids) as torch int64 CUDA tensors viewing the result's memory."""
        import torch
        a, b, n = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_int64()
        _check(load().dl_result_pairs(self._h, DL_MEM_DEVICE, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)),
               "dl_result_pairs")
        n = int(n.value)
        if n == 0:
            return (torch.empty(0, dtype=torch.int64, device="cuda"),) * 2
        return (torch.as_tensor(_DevView(a.value, n, "<i8", self), device="cuda"),
                torch.as_tensor(_DevView(b.value, n, "<i8", self), device="cuda"))

    def topk_host(self):
        """(ids [nq, k] int64, dist2 [nq, k] float64) numpy copies."""
        a, b = ctypes.c_void_p(), ctypes.c_void_p()
        k, nq = ctypes.c_int32(), ctypes.c_int64()
        _check(load().dl_result_topk(self._h, DL_MEM_HOST, ctypes.byref(a), ctypes.byref(b), ctypes.byref(k),
                                     ctypes.byref(nq)), "dl_result_topk")
        k, nq = int(k.value), int(nq.value)
        if k * nq == 0:
            return np.empty((nq, k), np.int64), np.empty((nq, k), np.float64)
        ids = np.ctypeslib.as_array(ctypes.cast(a, ctypes.POINTER(ctypes.c_int64)), shape=(nq, k)).copy()
        d2 = np.ctypeslib.as_array(ctypes.cast(b, ctypes.POINTER(ctypes.c_double)), shape=(nq, k)).copy()
        return ids, d2

    def free(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().dl_result_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def make_opts(precision="auto", self_mode="upper", out_capacity=0, stream=None, tile_n=0, timing=False,
              prune=False, cta_pair=0, epilogue_warps=0):
    o = dl_join_opts()
    load().dl_join_opts_default(ctypes.byref(o))
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.self_mode = DL_SELF_FULL if self_mode == "full" else DL_SELF_UPPER
    o.out_capacity = int(out_capacity)
    o.cuda_stream = _stream_handle(stream)
    o.tile_n = int(tile_n)
    o.timing = 1 if timing else 0
    o.prune = 1 if prune else 0
    o.cta_pair = int(cta_pair)
    o.epilogue_warps = int(epilogue_warps)
    return o


def color_hist(frames, boxes, bins, out=None, stream=None, timing=None):
    """dl_color_hist: float32 [n_boxes, br*bg*bb] histograms of the boxes {frame, x0, y0, x1, y1}
    of frames (a CUDA uint8 tensor [n_frames, H, W, 3]); boxes is a CUDA int32 tensor [n, 5].
    A dict passed as `timing` receives the counting kernel's event time ("count_ms")."""
    import torch
    assert frames.is_cuda and frames.dtype == torch.uint8 and frames.dim() == 4 and frames.shape[3] == 3
    frames = frames.contiguous()
    boxes = boxes.contiguous().to(device=frames.device, dtype=torch.int32)
    br, bg, bb = (int(b) for b in bins)
    nb = int(boxes.shape[0])
    if out is None:
        out = torch.empty((nb, br * bg * bb), dtype=torch.float32, device=frames.device)
    nF, H, W, _ = frames.shape
    ms = ctypes.c_float(0.0)
    rc = load().dl_color_hist(frames.data_ptr(), nF, H, W, boxes.data_ptr(), nb, br, bg, bb, out.data_ptr(),
                              ctypes.byref(ms) if timing is not None else None, _stream_handle(stream))
    _check(rc, "dl_color_hist")
    if timing is not None:
        timing["count_ms"] = float(ms.value)
    return out


def components(n: int, a, b, stream=None):
    """dl_components: (label int64 CUDA tensor [n], number of components) of the edges (a[e], b[e])."""
    import torch
    a = a.contiguous().to(dtype=torch.int64)
    b = b.contiguous().to(device=a.device, dtype=torch.int64)
    label = torch.empty(n, dtype=torch.int64, device=a.device)
    c = ctypes.c_int64()
    rc = load().dl_components(int(n), a.data_ptr(), b.data_ptr(), int(a.numel()), label.data_ptr(), ctypes.byref(c),
                              _stream_handle(stream))
    _check(rc, "dl_components")
    return label, int(c.value)


def dedup(X: Store, eps: float, labels=None, target: int = 0, plan="all", metric="l2", precision="auto",
          stream=None):
    """dl_dedup (q4): (component per caller row as an int64 CUDA tensor, number of distinct objects)."""
    import torch
    o = make_opts(precision, "upper", 0, stream, 0, False)
    comp = torch.empty(X.n, dtype=torch.int64, device="cuda")
    lab_ptr = None
    if labels is not None:
        labels = labels.contiguous().to(device="cuda", dtype=torch.int32)
        lab_ptr = labels.data_ptr()
    c = ctypes.c_int64()
    rc = load().dl_dedup(X.handle, METRICS[metric], float(eps), lab_ptr, int(target), DEDUP_PLANS[plan],
                         ctypes.byref(o), comp.data_ptr(), ctypes.byref(c))
    _check(rc, "dl_dedup")
    return comp, int(c.value)


def sim_join(R: Store, S: Store | None, eps: float, precision="auto", self_mode="upper", out_capacity=0,
             stream=None, tile_n=0, timing=False, allow_overflow=False, metric="l2", prune=False,
             cta_pair=0, epilogue_warps=0) -> Result:
    """dl_sim_join: every pair with canonical squared L2 distance <= eps^2; with
    metric="cosine" (stores from Store.normalized()) every pair with cosine >= eps; with
    metric="l1" / "chi2" every pair whose histogram distance is <= eps; with metric="ip"
    every pair whose canonical inner product is >= eps."""
    o = make_opts(precision, self_mode, out_capacity, stream, tile_n, timing, prune, cta_pair, epilogue_warps)
    h = ctypes.c_void_p()
    rc = load().dl_sim_join(R.handle, None if S is None else S.handle, METRICS[metric], float(eps),
                            ctypes.byref(o), ctypes.byref(h))
    if rc == DL_EOVERFLOW and allow_overflow:
        return Result(h)
    if h.value and rc != DL_OK:
        Result(h).free()
    _check(rc, "dl_sim_join")
    return Result(h)


def topk_join(Q: Store, S: Store, k: int, precision="auto", stream=None, timing=False, metric="l2", tile_n=0,
              epilogue_warps=0) -> Result:
    """dl_topk_join: the k nearest store rows of every query row, by (canonical D, row)."""
    o = make_opts(precision, "upper", 0, stream, tile_n, timing, epilogue_warps=epilogue_warps)
    h = ctypes.c_void_p()
    rc = load().dl_topk_join(Q.handle, S.handle, METRICS[metric], int(k), ctypes.byref(o), ctypes.byref(h))
    _check(rc, "dl_topk_join")
    return Result(h)


class BatchResult(Result):
    """A batch result: per-request pairs (eps requests) or top-k rows (top-k requests)."""

    def request_pairs(self, i: int):
        a, b, n = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_int64()
        _check(load().dl_result_request_pairs(self._h, i, DL_MEM_HOST, ctypes.byref(a), ctypes.byref(b),
                                              ctypes.byref(n)), "dl_result_request_pairs")
        n = int(n.value)
        if n == 0:
            return np.empty(0, np.int64), np.empty(0, np.int64)
        ra = np.ctypeslib.as_array(ctypes.cast(a, ctypes.POINTER(ctypes.c_int64)), shape=(n,)).copy()
        sa = np.ctypeslib.as_array(ctypes.cast(b, ctypes.POINTER(ctypes.c_int64)), shape=(n,)).copy()
        return ra, sa

    def request_topk(self, i: int):
        a, b = ctypes.c_void_p(), ctypes.c_void_p()
        k, nq = ctypes.c_int32(), ctypes.c_int64()
        _check(load().dl_result_request_topk(self._h, i, DL_MEM_HOST, ctypes.byref(a), ctypes.byref(b),
                                             ctypes.byref(k), ctypes.byref(nq)), "dl_result_request_topk")
        k, nq = int(k.value), int(nq.value)
        if k * nq == 0:
            return np.empty((nq, k), np.int64), np.empty((nq, k), np.float64)
        ids = np.ctypeslib.as_array(ctypes.cast(a, ctypes.POINTER(ctypes.c_int64)), shape=(nq, k)).copy()
        d2 = np.ctypeslib.as_array(ctypes.cast(b, ctypes.POINTER(ctypes.c_double)), shape=(nq, k)).copy()
        return ids, d2


def batch_join(S: Store, q_ids, q_feats, requests, stream=None, timing=False) -> BatchResult:
    """dl_batch_join. `requests` is a list of dicts {kind: 'eps'|'topk', q_begin, nq, eps | k}."""
    n = len(requests)
    arr = (dl_request * n)()
    for i, r in enumerate(requests):
        arr[i].kind = DL_REQ_TOPK if r["kind"] == "topk" else DL_REQ_EPS
        arr[i].k = int(r.get("k", 0) or 0)
        arr[i].eps = float(r.get("eps", 0.0) or 0.0)
        arr[i].q_begin = int(r["q_begin"])
        arr[i].nq = int(r["nq"])
    o = make_opts("auto", "upper", 0, stream, 0, timing)
    h = ctypes.c_void_p()
    if hasattr(q_feats, "data_ptr"):
        import torch
        q_feats = q_feats.contiguous().to(torch.float32)
        q_ids = q_ids.contiguous().to(device=q_feats.device, dtype=torch.int64)
        where = DL_MEM_DEVICE if q_feats.is_cuda else DL_MEM_HOST
        fp, ip = q_feats.data_ptr(), q_ids.data_ptr()
        nq_total, d = q_feats.shape
    else:
        q_feats = np.ascontiguousarray(q_feats, dtype=np.float32)
        q_ids = np.ascontiguousarray(q_ids, dtype=np.int64)
        where = DL_MEM_HOST
        fp, ip = q_feats.ctypes.data, q_ids.ctypes.data
        nq_total, d = q_feats.shape
    rc = load().dl_batch_join(S.handle, ip, fp, nq_total, d, where, arr, n, ctypes.byref(o), ctypes.byref(h))
    _check(rc, "dl_batch_join")
    return BatchResult(h)


class Server:
    """dl_server: a request loop with continuous batching over a resident store."""

    def __init__(self, S: Store, mem_budget_bytes: int = 8 << 30, slots: int = 2, max_batch_rows: int = 65536,
                 precision="auto"):
        self._store = S
        o = make_opts(precision, "upper", 0, 0, 0, False)
        h = ctypes.c_void_p()
        _check(load().dl_server_create(ctypes.byref(h), S.handle, int(mem_budget_bytes), int(slots),
                                       int(max_batch_rows), ctypes.byref(o)), "dl_server_create")
        self._h = h

    def submit(self, ids, feats, kind="eps", eps=0.0, k=0) -> int:
        feats = np.ascontiguousarray(feats, dtype=np.float32)
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        t = ctypes.c_uint64()
        rc = load().dl_submit(self._h, ids.ctypes.data, feats.ctypes.data, feats.shape[0],
                              DL_REQ_TOPK if kind == "topk" else DL_REQ_EPS, float(eps), int(k), ctypes.byref(t))
        _check(rc, "dl_submit")
        return int(t.value)

    def poll(self, ticket: int, timeout_us: int = 0):
        """Result when ready; None while pending (DL_EAGAIN / DL_ETIMEOUT); raises on other errors."""
        h = ctypes.c_void_p()
        rc = load().dl_poll(self._h, ctypes.c_uint64(ticket), int(timeout_us), ctypes.byref(h))
        if rc in (DL_EAGAIN, DL_ETIMEOUT):
            return None
        _check(rc, "dl_poll")
        return Result(h)

    def poll_status(self, ticket: int, timeout_us: int = 0):
        h = ctypes.c_void_p()
        rc = load().dl_poll(self._h, ctypes.c_uint64(ticket), int(timeout_us), ctypes.byref(h))
        return rc, (Result(h) if rc == DL_OK else None)

    def cancel(self, ticket: int) -> int:
        return int(load().dl_cancel(self._h, ctypes.c_uint64(ticket)))

    def stats(self) -> dict:
        st = dl_server_stats()
        _check(load().dl_server_get_stats(self._h, ctypes.byref(st)), "dl_server_get_stats")
        return {f: getattr(st, f) for f, _ in dl_server_stats._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().dl_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_wait_budget(clocks: int = 0):
    """dl_debug_set_wait_budget: SM-clock budget of the tensor-core kernels' bounded waits (0: default)."""
    _check(load().dl_debug_set_wait_budget(int(clocks)), "dl_debug_set_wait_budget")


def check_word() -> int:
    """dl_debug_check_word: the first failed bounds check of a checked build, (site << 40) | index; 0 = none."""
    w = ctypes.c_uint64()
    _check(load().dl_debug_check_word(ctypes.byref(w)), "dl_debug_check_word")
    return int(w.value)


def debug_scores(R: Store, S: Store, precision="bf16", stream=None):
    """(h~, E) as torch [|R|, |S|] float32 CUDA tensors: the kernel's h approximation and its bound."""
    import torch
    h = torch.empty(R.n, S.n, dtype=torch.float32, device="cuda")
    e = torch.empty(R.n, S.n, dtype=torch.float32, device="cuda")
    _check(load().dl_debug_scores(R.handle, S.handle, PRECISIONS[precision], h.data_ptr(), e.data_ptr(),
                                  _stream_handle(stream)), "dl_debug_scores")
    return h, e
