"""Sharded oracle evaluation for the full-size GPU tests (test infrastructure).

The store is written once to a temporary .npy that spawned worker processes
memory-map, so a multi-GB store is not pickled per task. Each task evaluates
single query rows against the whole store with the oracle: the rows within a
squared threshold (canonical FP64 distance <= e2), or the k nearest rows.
Workers are started with the spawn method, so a pool may be opened while the
calling process holds a CUDA context.
"""

from __future__ import annotations

import multiprocessing as mp
import os
import tempfile

import numpy as np

_S = None


def _init(path):
    global _S
    _S = np.load(path, mmap_mode="r")


def _within(task):
    import oracle
    q, e2 = task
    D = oracle.default().dist_block(q[None, :], _S)[0]
    return np.nonzero(D <= e2)[0].astype(np.int64)


def _topk(task):
    import oracle
    q, k = task
    idx, d2 = oracle.default().topk(q[None, :], _S, k)
    return idx[0], d2[0]


class OraclePool:
    def __init__(self, S: np.ndarray, procs: int | None = None):
        self._dir = tempfile.TemporaryDirectory()
        self._path = os.path.join(self._dir.name, "S.npy")
        np.save(self._path, np.ascontiguousarray(S, dtype=np.float32))
        n = procs or max(1, min(16, os.cpu_count() or 1))
        self._pool = mp.get_context("spawn").Pool(n, initializer=_init, initargs=(self._path,))

    def within(self, rows, e2s):
        """Async: per row, the store row indices with canonical D <= e2."""
        return self._pool.map_async(_within, [(np.asarray(q, np.float32), float(e)) for q, e in zip(rows, e2s)])

    def topk(self, rows, ks):
        """Async: per row, (indices [k], D64 [k]) of the k nearest store rows by (D64, row)."""
        return self._pool.map_async(_topk, [(np.asarray(q, np.float32), int(k)) for q, k in zip(rows, ks)])

    def close(self):
        self._pool.close()
        self._pool.join()
        self._dir.cleanup()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
