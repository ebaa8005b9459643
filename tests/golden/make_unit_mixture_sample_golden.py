"""Write the oracle's exact pair set for 16,384 sampled R rows of the 1M x 1M d=512 join.

The full R x S join of `rxs_unit_mixture_1m` (1,048,576 x 1,048,576 unit-norm d=512
rows) is too large for the oracle, so its exactness is checked on a seeded sample
of 16,384 R rows against ALL of S. This script runs the oracle (canonical FP64
nested loop, Sec. 5's join under the Euclidean threshold of Sec. 4) on that
sample, sharded over processes, and stores a digest:

  * sha256 of the sorted int64 pairs (sample position, S row), little-endian;
  * the per-sample-row match counts (uint16, zlib + base64), to localise a mismatch;
  * sha256 of the sampled R rows and of S (float32 bytes), so that a platform whose
    generator output differs is reported as such rather than as a join mismatch.

Only `oracle/` computes; the workload generator only draws inputs.

    python tests/golden/make_unit_mixture_sample_golden.py [procs]
"""

from __future__ import annotations

import base64
import hashlib
import json
import multiprocessing as mp
import os
import sys
import tempfile
import time
import zlib

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "unit_mixture_1m_sample16k.json")


def _shard(args):
    import oracle
    r_path, s_path, lo, hi, eps = args
    R = np.load(r_path, mmap_mode="r")
    S = np.load(s_path, mmap_mode="r")
    S = np.ascontiguousarray(S)
    o = oracle.default()
    out = []
    for a in range(lo, hi, 16):
        b = min(hi, a + 16)
        P = o.join(np.ascontiguousarray(R[a:b]), S, eps)
        P[:, 0] += a
        out.append(P)
    return np.concatenate(out, axis=0) if out else np.zeros((0, 2), np.int64)


def main(procs: int):
    from paper_1812_07607_gb300 import workloads as W
    t0 = time.time()
    wl = W.rxs_unit_mixture_1m()
    rows = W.sample_rows(wl.R.shape[0], W.UNIT_MIXTURE_SAMPLE_ROWS, W.UNIT_MIXTURE_SAMPLE_SEED)
    Rs = np.ascontiguousarray(wl.R[rows])
    print(f"generated in {time.time() - t0:.0f} s; eps {wl.eps!r}", file=sys.stderr)
    with tempfile.TemporaryDirectory() as td:
        rp, sp = os.path.join(td, "R.npy"), os.path.join(td, "S.npy")
        np.save(rp, Rs)
        np.save(sp, wl.S)
        n = Rs.shape[0]
        step = 256
        jobs = [(rp, sp, a, min(n, a + step), wl.eps) for a in range(0, n, step)]
        with mp.get_context("spawn").Pool(procs) as pool:
            parts = pool.map(_shard, jobs)
    P = np.concatenate(parts, axis=0)
    P = P[np.lexsort((P[:, 1], P[:, 0]))]
    counts = np.bincount(P[:, 0], minlength=Rs.shape[0]).astype(np.uint16)
    rec = {
        "workload": "rxs_unit_mixture_1m",
        "eps": wl.eps,
        "sample_seed": W.UNIT_MIXTURE_SAMPLE_SEED,
        "sample_rows": int(Rs.shape[0]),
        "pairs": int(P.shape[0]),
        "pairs_sha256": hashlib.sha256(np.ascontiguousarray(P, dtype="<i8").tobytes()).hexdigest(),
        "counts_zlib_b64": base64.b64encode(zlib.compress(counts.astype("<u2").tobytes(), 9)).decode(),
        "r_sample_sha256": hashlib.sha256(Rs.astype("<f4").tobytes()).hexdigest(),
        "s_sha256": hashlib.sha256(np.ascontiguousarray(wl.S, dtype="<f4").tobytes()).hexdigest(),
        "command": "python tests/golden/make_unit_mixture_sample_golden.py",
    }
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(f"{P.shape[0]} pairs in {time.time() - t0:.0f} s -> {OUT}", file=sys.stderr)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1))
