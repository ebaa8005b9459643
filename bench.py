"""Benchmark: exact epsilon-join throughput (Gpairs/s) on one or more GB300s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (default): self-join of 262,144 patches with d=128 colour-histogram
features (8,192 Dirichlet(0.5) centroids + N(0, 0.01^2) jitter, clipped and
renormalised; eps calibrated for ~20 matches per patch), synthetic and seeded.
A step is one dl_sim_join call on the resident store -- the tensor-core pass,
the exact recheck of the band pairs and the id-pair write-out -- and the metric
is the N(N-1)/2 pairs it is defined over divided by the step time.

Rank 0 prints one JSON line. With N > 1 (torchrun), every rank joins its own
replica of the workload (the join has no cross-rank exchange) and the value is
all ranks' pairs over the slowest rank's time.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact eps-join pair-distances/sec"
UNIT = "Gpairs/s"
SEED_BATCH = 1812076074
SEED_SERVE = 1812076075
L2_FLUSH_BYTES = 512 << 20      # > 129 MB L2
_KEEP = {}                      # workloads the GPU legs generated, reused by the oracle samples


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU-oracle sample")
    ap.add_argument("--no-baselines", action="store_true", help="skip the plain-FP32 and CPU legs")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-requests leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-precision", action="store_true", help="skip the d=512 BF16 / FP8 leg")
    ap.add_argument("--no-rows", action="store_true",
                    help="skip the colour-histogram, L1 / chi-square and dedup leg")
    ap.add_argument("--profile-case", choices=sorted(PROFILE_CASES), default=None,
                    help="run one small profiling case --profile-calls times and print its timings (no bench line)")
    ap.add_argument("--profile-calls", type=int, default=3,
                    help="calls of the profiling case (the first calls of a shape class are autotuner trials)")
    ap.add_argument("--peak-probe", action="store_true",
                    help="measure the BF16 and FP8 e4m3 cuBLAS GEMM peaks of this GPU and print them (no bench line)")
    ap.add_argument("--no-latency", action="store_true", help="skip the 2,000 x 2,000 latency leg")
    ap.add_argument("--serving-seconds", type=float, default=4.0)
    ap.add_argument("--serving-rate", type=float, default=2000.0, help="Poisson arrival rate, requests/s")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def fp8_peak():
    """The FP8 e4m3 GEMM peak measured on this GPU model by `bench.py --peak-probe` (TFLOP/s), or None."""
    p = os.path.join(ROOT, "profiles", "fp8_e4m3_peak_gb300.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        return json.load(f).get("fp8_peak_tflops")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return {"bf16_tflops": j.get("bf16_tflops"), "bf16_tflops_sustained": j.get("bf16_tflops_sustained"),
                "hbm_gbs": j.get("hbm_gbs"), "source": "measured"}
    return {"bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "hbm_gbs": 6800.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [r.split(", ") for r in self.tmp.read().strip().splitlines() if r.strip()]
        os.unlink(self.tmp.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip() == "Active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate(total_ms: float, pairs_per_step: int, steps: int, world: int, device=None):
    """Whole-job throughput: all ranks' pairs over the slowest rank's timed total (Gpairs/s).

    With world > 1 the per-rank totals are reduced with MAX over the process group.
    Returns (value, max_total_ms).
    """
    if world > 1:
        import torch
        import torch.distributed as tdist
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world * pairs_per_step * steps / (total_ms / 1e3) / 1e9, total_ms


def load_workload(rank: int):
    from paper_1812_07607_gb300 import workloads as W
    return W.self_clustered_262k()


def traffic_record():
    """DRAM bytes per launch of the join kernel from the committed ncu summary, if still current."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "tc_join_kernel_self_clustered_262k.json")
    src = os.path.join(ROOT, "paper_1812_07607_gb300", "csrc", "join_tc.cu")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()
    return rec.get("dram_bytes_per_launch") if rec.get("join_tc_sha256") == h else None


def cpu_oracle_rate(wl, budget_s: float):
    """Pairs/s of the FP64 CPU oracle (single thread) on a bounded sample of the workload."""
    import oracle
    orc = oracle.default()
    R = wl.R
    n = R.shape[0]
    eps = wl.eps
    t0 = time.perf_counter()
    orc.join(R[:4], R, eps, oracle.MODE_RXS)
    dt = time.perf_counter() - t0
    per_row = max(dt / 4, 1e-6)
    rows = int(max(4, min(n, budget_s / per_row)))
    t0 = time.perf_counter()
    orc.join(R[4:4 + rows], R, eps, oracle.MODE_RXS)
    dt = time.perf_counter() - t0
    pairs = rows * n
    return pairs / dt / 1e9, {"rows": rows, "pairs": pairs, "seconds": round(dt, 3)}


def host_cpu():
    """(cores this process may run on, CPU model name)."""
    import platform
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return cores, model or platform.machine()


def _oracle_warm(_):
    """Spawned worker: import and load the oracle before the timed region."""
    import oracle
    oracle.default()
    time.sleep(0.3)   # so that every worker of the pool takes one warm-up task
    return os.getpid()


def _oracle_shard(task):
    """Spawned worker: rows [r0, r1) of the memory-mapped store against all of it, FP64 oracle."""
    import oracle
    path, r0, r1, eps = task
    X = np.load(path, mmap_mode="r")
    t0 = time.perf_counter()
    oracle.default().join(np.ascontiguousarray(X[r0:r1]), X, eps, oracle.MODE_RXS)
    return time.perf_counter() - t0


def cpu_oracle_all_cores(wl, per_row_s: float, budget_s: float):
    """The same single-threaded FP64 oracle on every host core at once: one spawned process per
    core, each on its own shard of query rows against the whole store (the result does not
    depend on the split). Returns (Gpairs/s over the wall time of all shards, info)."""
    import multiprocessing as mp
    cores, model = host_cpu()
    n = wl.R.shape[0]
    rows_each = int(max(1, min(n // cores, budget_s / max(per_row_s, 1e-6))))
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "R.npy")
        np.save(path, wl.R)
        with mp.get_context("spawn").Pool(cores) as pool:
            # bounded waits: a pool whose workers cannot start would otherwise wait forever
            pool.map_async(_oracle_warm, range(cores), chunksize=1).get(timeout=120)
            tasks = [(path, i * rows_each, (i + 1) * rows_each, wl.eps) for i in range(cores)]
            t0 = time.perf_counter()
            worker_s = pool.map_async(_oracle_shard, tasks, chunksize=1).get(timeout=30 * budget_s + 120)
            dt = time.perf_counter() - t0
    pairs = cores * rows_each * n
    return pairs / dt / 1e9, {"cores": cores, "cpu_model": model, "rows": cores * rows_each, "pairs": pairs,
                              "seconds": round(dt, 3), "slowest_shard_s": round(max(worker_s), 3)}


def cpu_oracle_configs(budget_s: float = 3.0):
    """The FP64 oracle (one thread) on the other configs: the 2,000 x 2,000 join in full, and a
    bounded slice of query rows x the whole store for the precision, batching and serving
    workloads (reusing the inputs their GPU legs generated; a config whose leg did not run is
    skipped)."""
    import oracle
    from paper_1812_07607_gb300 import workloads as W
    orc = oracle.default()
    out = {}
    c1 = W.rxs_histograms_2k()
    t0 = time.perf_counter()
    n1 = len(orc.join(c1.R, c1.S, c1.eps, oracle.MODE_RXS))
    dt = time.perf_counter() - t0
    out["rxs_histograms_2k"] = {"value": c1.pairs / dt / 1e9, "unit": UNIT, "seconds": round(dt, 4),
                                "pairs_out": n1, "sample": "the whole 2,000 x 2,000 join, d=64"}
    cases = []
    if "precision" in _KEEP:
        wl = _KEEP["precision"]
        cases.append(("rxs_unit_mixture_1m", wl.R, wl.S, wl.eps))
    if "batch" in _KEEP:
        st, Q, table = _KEEP["batch"]
        cases.append(("batch_store_2m", Q, st.X, W.eps_for_selectivity(table, 2e-3)))
    if "serve" in _KEEP:
        sw = _KEEP["serve"]
        cases.append(("serve_store_4m", sw.queries(64, SEED_SERVE + 99), sw.X, W.eps_for_selectivity(sw.eps_table(), 2e-3)))
    for name, Q, S, eps in cases:
        t0 = time.perf_counter()
        orc.join(Q[:1], S, eps, oracle.MODE_RXS)
        per_row = time.perf_counter() - t0
        rows = int(max(1, min(Q.shape[0] - 1, budget_s / max(per_row, 1e-6))))
        t0 = time.perf_counter()
        orc.join(Q[1:1 + rows], S, eps, oracle.MODE_RXS)
        dt = time.perf_counter() - t0
        out[name] = {"value": rows * S.shape[0] / dt / 1e9, "unit": UNIT, "seconds": round(dt, 3),
                     "sample": f"{rows} query rows x all {S.shape[0]} store rows, d={S.shape[1]}",
                     "s_per_query_row": round(dt / rows, 4)}
    return out


def cpu_oracle_rows(W):
    """The FP64 CPU oracle (one thread) on bounded samples of the further rows' workloads, in
    the units of their GPU figures. Inputs come from the generators only."""
    import oracle
    orc = oracle.default()
    out = {"cores": 1, "kind": "oracle"}
    wl = W.traffic_boxes_1080p()
    boxes = wl.boxes[:512]
    px = int(((boxes[:, 3] - boxes[:, 1]).astype(np.int64) * (boxes[:, 4] - boxes[:, 2])).sum())
    t0 = time.perf_counter()
    orc.color_hist(wl.frames, boxes, wl.bins)
    dt = time.perf_counter() - t0
    out["color_hist"] = {"value": (3 * px + 4 * 128 * len(boxes)) / dt / 1e9, "unit": "GB/s",
                         "sample": f"the first {len(boxes)} boxes ({px} pixels), {dt:.3f} s"}
    X, thr = W.hist_clustered_64k()
    for name, metric in (("l1", oracle.METRIC_L1), ("chi2", oracle.METRIC_CHI2)):
        t0 = time.perf_counter()
        orc.hist_join(X[:16], X, thr[name], metric, oracle.MODE_RXS)
        dt = time.perf_counter() - t0
        out[name] = {"value": 16 * X.shape[0] / dt / 1e9, "unit": "Gpairs/s",
                     "sample": f"16 rows x all {X.shape[0]} rows, {dt:.3f} s"}
    wl2 = W.self_clustered_262k()
    Y = np.ascontiguousarray(wl2.R[:4096])
    t0 = time.perf_counter()
    _, c = orc.dedup(Y, wl2.eps)
    dt = time.perf_counter() - t0
    out["dedup"] = {"value": 4096 / dt, "unit": "rows/s", "distinct": c,
                    "sample": f"the first 4,096 rows: self-join (8.4 M pairs) and components, {dt:.3f} s"}
    return out


def batch_leg(dl, seed=SEED_BATCH, n_req=4096, reps=2):
    """The batching config: 4,096 eps / top-k requests in ONE dl_batch_join on the 2,097,152 x 128 store.

    Request sizes lognormal(5, 1.5) clipped to [1, 8192]; 70% eps-joins at a selectivity
    uniform in [0.05%, 0.5%] of the store (eps from the oracle-calibrated table), 30% top-k
    with k = 10; queries are fresh jitters of the store's centroids, resident on the device.
    Throughput counts pairs evaluated (query rows x store rows) per second of the whole call.
    """
    import torch
    from paper_1812_07607_gb300 import workloads as W
    st = W.batch_store_2m()
    g = W.rng(seed)
    reqs = W.request_mix(g, n_req, 5.0, 1.5, 8192, topk_frac=0.3, ks=(10,), sel_lo=5e-4, sel_hi=5e-3)
    table = st.eps_table()
    off = 0
    for r in reqs:
        r["q_begin"] = off
        off += r["nq"]
        if r["kind"] == "eps":
            r["eps"] = W.eps_for_selectivity(table, r["selectivity"])
    Q = st.queries(off, seed + 1)
    _KEEP["batch"] = (st, Q, table)
    store = dl.Store(torch.from_numpy(st.ids).cuda(), torch.from_numpy(st.X).cuda())
    Qd = torch.from_numpy(Q).cuda()
    qd = torch.arange(off, dtype=torch.int64).cuda()
    times, stats, out_pairs = [], None, 0
    warm = 4   # the tile autotuner's trial calls (ε rows 2 candidates + 1, top-k 3 + 1; the first also sizes buffers)
    for i in range(warm + reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = dl.batch_join(store, qd, Qd, reqs, timing=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        stats = res.stats()
        out_pairs = res.count()
        res.free()
        if i >= warm:
            times.append(dt)
    store.close()
    t = statistics.median(times)
    pairs = off * st.X.shape[0]
    return {"value": pairs / t / 1e9, "unit": UNIT, "ms_per_batch": 1e3 * t, "requests": n_req,
            "requests_per_s": n_req / t, "query_rows": off, "pairs_evaluated": pairs, "pairs_out": out_pairs,
            "band_pairs": stats["band_pairs"], "fp64_pairs": stats["fp64_pairs"],
            "ms_eps_contraction": stats["ms_main"], "ms_eps_decide_scatter": stats["ms_recheck"],
            "tile_n": stats["tile_n"], "cta_pair": stats["cta_pair"], "epilogue_warps": stats["epilogue_warps"],
            "ms_device_total": stats["ms_total"],
            "config": "batch_store_2m: 2,097,152 x 128 store; 4,096 requests in one call, sizes lognormal(5,1.5) "
                      "in [1,8192]; 70% eps at selectivity U[0.05%,0.5%], 30% top-k k=10; device inputs"}


def serving_leg(dl, seconds=4.0, rates=(2000.0, 1000.0, 500.0), seed=SEED_SERVE):
    """The serving config: Poisson arrivals into the request loop over the 4,194,304 x 256 store.

    70% eps-joins (selectivity U[0.05%, 0.5%]) and 30% top-k with k uniform over
    {1, 10, 100}; query sizes lognormal(4, 1.5) clipped to [1, 4096]; submit-to-ready
    latency p50/p99 and completed requests per second at each offered rate (the first
    rate is the serving config's; the others are the sweep below it).
    """
    import torch
    from paper_1812_07607_gb300 import workloads as W
    sw = W.serve_store_4m()
    _KEEP["serve"] = sw
    store = dl.Store(torch.from_numpy(sw.ids).cuda(), torch.from_numpy(sw.X).cuda())
    # warm-up at the first rate (not reported): the first batches of each shape class are the
    # tile autotuner's trial calls, and the first calls size the library's buffers
    _serve_once(dl, W, sw, store, min(2.0, seconds), rates[0], seed + 1000)
    out = None
    sweep = []
    for i, rate in enumerate(rates):
        r = _serve_once(dl, W, sw, store, seconds, rate, seed + 10 * i)
        sweep.append({k: r[k] for k in ("offered_req_per_s", "req_per_s", "p50_ms", "p99_ms", "max_ms", "batches")})
        if out is None:
            out = r
    store.close()
    out["sweep"] = sweep
    return out


def _serve_once(dl, W, sw, store, seconds, rate, seed):
    import threading
    g = W.rng(seed)
    n = int(seconds * rate)
    reqs = W.request_mix(g, n, 4.0, 1.5, 4096, topk_frac=0.3, ks=(1, 10, 100), sel_lo=5e-4, sel_hi=5e-3)
    table = sw.eps_table()
    arrivals = np.cumsum(g.exponential(1.0 / rate, size=n))
    total = sum(r["nq"] for r in reqs)
    Q = sw.queries(total, seed + 1)
    sv = dl.Server(store, mem_budget_bytes=64 << 30, slots=3, max_batch_rows=65536)
    tickets = []
    lock = threading.Lock()

    def submitter():
        off = 0
        t0 = time.perf_counter()
        for i, r in enumerate(reqs):
            while time.perf_counter() - t0 < arrivals[i]:
                time.sleep(5e-5)
            q = Q[off:off + r["nq"]]
            ids = np.arange(off, off + r["nq"], dtype=np.int64)
            off += r["nq"]
            if r["kind"] == "eps":
                t = sv.submit(ids, q, "eps", eps=W.eps_for_selectivity(table, r["selectivity"]))
            else:
                t = sv.submit(ids, q, "topk", k=r["k"])
            with lock:
                tickets.append(t)

    th = threading.Thread(target=submitter)
    t_start = time.perf_counter()
    th.start()
    got = 0
    while got < n:
        with lock:
            pend = tickets[got:]
        if not pend:
            time.sleep(1e-4)
            continue
        res = sv.poll(pend[0], timeout_us=200_000)
        if res is None:
            continue
        res.free()
        got += 1
    wall = time.perf_counter() - t_start
    th.join()
    st = sv.stats()
    sv.close()
    pairs = total * sw.X.shape[0]
    return {"offered_req_per_s": rate, "requests": n, "seconds": wall, "completed": st["completed"],
            "req_per_s": st["completed"] / wall, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "max_ms": st["max_ms"], "pairs_per_s_G": pairs / wall / 1e9, "batches": st["batches"],
            "mean_batch_requests": st["mean_batch_requests"],
            "config": "serve_store_4m: 4,194,304 x 256 store resident; Poisson arrivals; 70% eps at selectivity "
                      "U[0.05%,0.5%] / 30% top-k k in {1,10,100}; sizes lognormal(4,1.5) in [1,4096]; "
                      "3 stream slots; results stay on the device until polled"}


def precision_leg(dl, reps=2):
    """The precision config: the 1,048,576 x 1,048,576 d=512 unit-norm R x S join, BF16 and FP8 e4m3."""
    import torch
    from paper_1812_07607_gb300 import workloads as W
    wl = W.rxs_unit_mixture_1m()
    _KEEP["precision"] = wl
    n = wl.R.shape[0]
    S = dl.Store(torch.arange(n).cuda(), torch.from_numpy(wl.S).cuda())
    R = dl.Store(torch.arange(n).cuda(), torch.from_numpy(wl.R).cuda())
    out = {"config": "rxs_unit_mixture_1m: 1,048,576 x 1,048,576, d=512 unit-norm, 4,096-component mixture; "
                     "exact pair set (parity: 16,384 sampled rows against the oracle digest)",
           "pairs_evaluated": n * n}
    for prec in ("bf16", "fp8"):
        ts, st = [], None
        warm = 5 if prec == "bf16" else 4   # the tile autotuner's trial calls (4 candidates BF16, 3 FP8, + 1)
        for i in range(warm + reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = dl.sim_join(R, S, wl.eps, precision=prec, timing=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            st = res.stats()
            res.free()
            if i >= warm:
                ts.append(dt)
        t = statistics.median(ts)
        tflops = 2.0 * 512 * n * n / (st["ms_main"] / 1e3) / 1e12
        pk = peaks()["bf16_tflops"] if prec == "bf16" else fp8_peak()
        out[prec] = {"value": n * n / t / 1e9, "unit": UNIT, "ms": 1e3 * t, "ms_main": st["ms_main"],
                     "ms_recheck": st["ms_recheck"], "band_pairs": st["band_pairs"], "fp64_pairs": st["fp64_pairs"],
                     "pairs_out": st["pairs_out"], "tile_n": st["tile_n"], "main_tflops": tflops,
                     "main_frac_of_measured_peak": (tflops / pk) if pk else None,
                     "peak_tflops": pk, "peak_source": ("MEASURED_PEAKS.json bf16 burst" if prec == "bf16"
                                                        else "profiles/fp8_e4m3_peak_gb300.json (bench.py --peak-probe)")}
    R.close()
    S.close()
    return out


def latency_leg(dl, reps=50):
    """The 2,000 x 2,000 d=64 R x S join (4e6 pairs, ~0.1% selectivity): too small to fill the GPU,
    so it is reported as per-call latency -- host wall time of dl_sim_join on resident stores,
    including the synchronisation that returns the pair count."""
    import torch
    from paper_1812_07607_gb300 import workloads as W
    wl = W.rxs_histograms_2k()
    R = dl.Store(torch.from_numpy(wl.r_ids).cuda(), torch.from_numpy(wl.R).cuda())
    S = dl.Store(torch.from_numpy(wl.s_ids).cuda(), torch.from_numpy(wl.S).cuda())
    out = {"config": "rxs_histograms_2k: 2,000 x 2,000, d=64 Dirichlet(0.5) histograms, eps at 0.1% selectivity"}
    for prec in ("bf16", "fp32"):
        for _ in range(6):   # warm-up, including the tile autotuner's trial calls (4 candidates + 1)
            dl.sim_join(R, S, wl.eps, precision=prec).free()
        ts, n = [], 0
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = dl.sim_join(R, S, wl.eps, precision=prec)
            n = res.count()
            ts.append(1e3 * (time.perf_counter() - t0))
            res.free()
        ts.sort()
        p50 = statistics.median(ts)
        out[prec] = {"p50_ms": p50, "p99_ms": ts[min(len(ts) - 1, int(0.99 * len(ts)))], "pairs_out": n,
                     "value": wl.pairs / (p50 / 1e3) / 1e9, "unit": UNIT}
    R.close()
    S.close()
    return out


def peak_probe(seconds: float = 4.0, n: int = 8192):
    """Dense tensor-core peaks of this GPU measured through cuBLAS: BF16 (torch.matmul) and FP8
    e4m3 (torch._scaled_mm, unit scales, BF16 out), n^3 GEMMs counted as 2 n^3 flops. Burst = best
    of 10 CUDA-event timings; sustained = back-to-back calls for `seconds`. A calibration of the
    denominators, not a kernel of this library."""
    import torch
    torch.manual_seed(0)
    a16 = torch.randn(n, n, device="cuda", dtype=torch.bfloat16)
    b16 = torch.randn(n, n, device="cuda", dtype=torch.bfloat16)
    a8 = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
    b8 = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn).t()   # column-major operand
    one = torch.ones((), device="cuda", dtype=torch.float32)
    fns = {"bf16": lambda: torch.matmul(a16, b16),
           "fp8_e4m3": lambda: torch._scaled_mm(a8, b8, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)}
    flops = 2.0 * n ** 3
    st = torch.cuda.current_stream()
    sampler = ClockSampler(torch.cuda.current_device())
    out = {"n": n, "method": f"{n}^3 GEMM, 2n^3 flops; burst: best of 10 (CUDA events); sustained: "
                             f"back to back for {seconds} s"}
    sampler.start()
    for name, f in fns.items():
        for _ in range(3):
            f()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            f()
            e1.record(st)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        calls = max(10, int(seconds / (best / 1e3)))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(calls):
            f()
        e1.record(st)
        e1.synchronize()
        out[name] = {"burst_tflops": flops / (best / 1e3) / 1e12,
                     "sustained_tflops": flops * calls / (e0.elapsed_time(e1) / 1e3) / 1e12}
    out["clocks"] = sampler.stop()
    return out


def _event_ms(fn, reps, flush=None):
    """Median CUDA-event time (ms) of fn() on the current stream over reps calls after one warm call;
    flush() (outside the events) runs before each timed call."""
    import torch
    st = torch.cuda.current_stream()
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        fn()
        b.record(st)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def rows_leg(dl, sm_mhz=None, reps=5):
    """The further rows: the colour-histogram transformer, the L1 / chi-square self-joins, the
    inner-product join, the pruned join and q4 deduplication, each on its own seeded workload at
    full size (parity in the GPU tests)."""
    import torch
    from paper_1812_07607_gb300 import workloads as W
    pk = peaks()
    mhz = sm_mhz or 2070.0
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    scratch = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    flush = lambda: scratch.fill_(1)   # noqa: E731  (512 MiB > L2)
    out = {"clock_mhz_for_alu_peaks": mhz}

    wl = W.traffic_boxes_1080p()
    fr = torch.from_numpy(wl.frames).cuda()
    bx = torch.from_numpy(wl.boxes).cuda()
    d = wl.bins[0] * wl.bins[1] * wl.bins[2]
    h = torch.empty((len(wl.boxes), d), dtype=torch.float32, device="cuda")
    kms = []

    def hist_call():
        tm = {}
        dl.color_hist(fr, bx, wl.bins, out=h, timing=tm)
        kms.append(tm["count_ms"])

    ms = _event_ms(hist_call, reps, flush)
    kern = statistics.median(kms[1:])
    byt = 3 * wl.pixels + 4 * h.numel()
    out["color_hist"] = {
        "config": f"traffic_boxes_1080p: {fr.shape[0]} frames 1920x1080 RGB8, {len(wl.boxes)} detector boxes, "
                  f"bins {wl.bins} (d={d}); L2 flushed between calls",
        "ms_call": ms, "ms_count_kernel": kern, "patches_per_s": len(wl.boxes) / (ms / 1e3), "pixels": wl.pixels,
        "call_GBps": byt / (ms / 1e3) / 1e9,
        "roofline": {"bound": "hbm", "achieved": byt / (kern / 1e3) / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": byt / (kern / 1e3) / 1e9 / pk["hbm_gbs"], "kernel": "k_hist_count",
                     "algorithmic": f"3 B/pixel x {wl.pixels} + 4 B x {h.numel()} bins = {byt} B per launch"}}
    del fr, bx, h

    X, thr = W.hist_clustered_64k()
    n = X.shape[0]
    Xs = dl.Store(torch.arange(n, device="cuda"), torch.from_numpy(X).cuda())
    P = n * (n - 1) // 2
    for metric, unit_ops, lanes, what in (("l1", 2, 128, "FP32 add (sub, add |t|) per term, 128 lanes/SM"),
                                          ("chi2", 1, 16, "one MUFU reciprocal per term, 16 lanes/SM")):
        st = {}

        def call():
            r = dl.sim_join(Xs, None, thr[metric], metric=metric, timing=True)
            st.update(r.stats())
            r.free()

        ms = _event_ms(call, 3)
        ops = unit_ops * X.shape[1] * P
        kern_ms = st["ms_main"]
        peak = sms * lanes * mhz * 1e6
        out[metric] = {"config": f"hist_clustered_64k: {n} x d=128 clustered histograms, self-join, "
                                 f"eps={thr[metric]:.6g} (20 matches per row)",
                       "value": P / (ms / 1e3) / 1e9, "unit": "Gpairs/s", "ms": ms, "ms_main": kern_ms,
                       "pairs_out": st["pairs_out"], "band_pairs": st["band_pairs"], "fp64_pairs": st["fp64_pairs"],
                       "roofline": {"bound": "alu", "achieved": ops / (kern_ms / 1e3) / 1e12,
                                    "peak": peak / 1e12, "unit": "Tops/s", "frac": ops / (kern_ms / 1e3) / peak,
                                    "algorithmic": f"{unit_ops} x d x {P} pairs ({what}), at {mhz:.0f} MHz"}}
    # top-10 under each histogram distance: 4,096 query rows against the same store
    for metric in ("l1", "chi2"):
        Qs = dl.Store(torch.arange(4096, device="cuda"), torch.from_numpy(X[:4096]).cuda())

        def call_tk():
            dl.topk_join(Qs, Xs, 10, metric=metric).free()

        ms = _event_ms(call_tk, 3)
        out[metric + "_topk10"] = {"config": f"4,096 query rows x hist_clustered_64k ({n} x d=128), k=10",
                                   "value": 4096 * n / (ms / 1e3) / 1e9, "unit": "Gpairs/s", "ms": ms}
        Qs.close()
    Xs.close()

    # the inner-product threshold join on rows of any norm (BF16 tensor cores, exact)
    g = W.rng(W.SEED_BASE + 120)
    nip, dip = 65536, 128
    Rip = (g.standard_normal((nip, dip)) * 2.0 ** g.uniform(-1.0, 1.0, (nip, 1))).astype(np.float32)
    Sip = (g.standard_normal((nip, dip)) * 2.0 ** g.uniform(-1.0, 1.0, (nip, 1))).astype(np.float32)
    t_ip = float(np.quantile(Rip[:256].astype(np.float64) @ Sip.astype(np.float64).T, 1.0 - 5e-4))
    Rs_ip = dl.Store(torch.arange(nip, device="cuda"), torch.from_numpy(Rip).cuda())
    Ss_ip = dl.Store(torch.arange(nip, device="cuda") + nip, torch.from_numpy(Sip).cuda())
    st = {}

    def call_ip():
        r = dl.sim_join(Rs_ip, Ss_ip, t_ip, metric="ip", timing=True)
        st.update(r.stats())
        r.free()

    call_ip()   # the autotuner's trials of this shape class
    for _ in range(4):
        call_ip()
    ms = _event_ms(call_ip, reps)
    P = nip * nip
    kern_ms = st["ms_main"]
    out["inner_product"] = {"config": f"{nip} x {nip}, d={dip} signed rows of norms spanning a factor 4, "
                                      f"t at the 0.9995 quantile of q.x ({t_ip:.6g})",
                            "value": P / (ms / 1e3) / 1e9, "unit": "Gpairs/s", "ms": ms, "ms_main": kern_ms,
                            "pairs_out": st["pairs_out"], "band_pairs": st["band_pairs"],
                            "fp64_pairs": st["fp64_pairs"],
                            "roofline": {"bound": "tensor", "achieved": 2.0 * dip * P / (kern_ms / 1e3) / 1e12,
                                         "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                                         "frac": 2.0 * dip * P / (kern_ms / 1e3) / 1e12 / pk["bf16_tflops"],
                                         "kernel": "tc_join_kernel<256> (BF16, zero column term)"}}
    Rs_ip.close()
    Ss_ip.close()
    del Rip, Sip

    # the exact pruned join on tracked objects: dense join, store clustering (one-time), pruned join
    wt = W.tracked_objects_262k()
    nt_ = wt.R.shape[0]
    St = dl.Store(torch.from_numpy(wt.r_ids).cuda(), torch.from_numpy(wt.R).cuda())
    Pt = nt_ * (nt_ - 1) // 2
    dst, pst = {}, {}

    def dense_call():
        r = dl.sim_join(St, None, wt.eps, precision="bf16", timing=True)
        dst.update(r.stats())
        r.free()

    for _ in range(5):   # the tile autotuner's trial calls (4 candidates + 1)
        dense_call()
    ms_dense = _event_ms(dense_call, 3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Ct = St.clustered(1024, iters=5)
    torch.cuda.synchronize()
    ms_cluster = 1e3 * (time.perf_counter() - t0)

    def pruned_call():
        r = dl.sim_join(Ct, None, wt.eps, precision="bf16", timing=True, prune=True)
        pst.update(r.stats())
        r.free()

    ms_pruned = _event_ms(pruned_call, 3)
    assert pst["pairs_out"] == dst["pairs_out"]
    out["pruned_join"] = {
        "config": f"tracked_objects_262k: {nt_} x d=128 histograms of 256 tracked objects, self-join, "
                  f"eps={wt.eps:.6g} (100 matches per row); store clustered by 5 k-means iterations, 1,024 centres",
        "dense": {"value": Pt / (ms_dense / 1e3) / 1e9, "unit": "Gpairs/s", "ms": ms_dense,
                  "ms_main": dst["ms_main"], "pairs_out": dst["pairs_out"]},
        "pruned": {"value": Pt / (ms_pruned / 1e3) / 1e9, "unit": "Gpairs/s (pairs of the join / time)",
                   "ms": ms_pruned, "ms_main": pst["ms_main"], "pairs_out": pst["pairs_out"],
                   "tile_pairs": pst["tile_pairs"], "tile_pairs_kept": pst["tile_pairs_kept"]},
        "cluster_store_ms": ms_cluster,
        "speedup": ms_dense / ms_pruned}
    Ct.close()
    St.close()

    wl2 = W.self_clustered_262k()
    labels = torch.from_numpy(W.object_labels(W.rng(W.SEED_BASE + 107), wl2.groups, 8192)).cuda()
    S = dl.Store(torch.from_numpy(wl2.r_ids).cuda(), torch.from_numpy(wl2.R).cuda())
    dd = {"config": "self_clustered_262k + object labels (0 person / 1 vehicle / 2 other per object, 8% "
                    "detector flips); target label 0; eps of the store (mean 20 matches)"}
    for plan in ("all", "filter_match", "match_filter"):
        cnt = []
        ms = _event_ms(lambda: cnt.append(dl.dedup(S, wl2.eps, labels, 0, plan=plan)[1]), 3)
        dd[plan] = {"ms": ms, "distinct": cnt[-1]}
    r = dl.sim_join(S, None, wl2.eps)
    a, b = (torch.as_tensor(v) for v in r.pairs_device())
    ids = torch.from_numpy(wl2.r_ids).cuda()
    srt, perm = torch.sort(ids)
    ra, rb = perm[torch.searchsorted(srt, a)], perm[torch.searchsorted(srt, b)]
    ms = _event_ms(lambda: dl.components(wl2.R.shape[0], ra, rb), reps)
    dd["components"] = {"ms": ms, "edges": int(ra.numel()), "edges_per_s": ra.numel() / (ms / 1e3)}
    r.free()
    S.close()
    out["dedup"] = dd
    del scratch
    try:
        out["cpu_baseline"] = cpu_oracle_rows(W)
    except Exception as exc:   # the CPU figures are context; never lose the GPU ones for them
        out["cpu_baseline"] = {"error": repr(exc)[:200]}
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    wl = load_workload(0)
    import oracle
    orc = oracle.default()
    n = wl.R.shape[0]
    t0 = time.perf_counter()
    orc.join(wl.R[:2], wl.R, wl.eps, oracle.MODE_RXS)
    per_row = (time.perf_counter() - t0) / 2
    step_budget = max(0.5, min(6.0, 150.0 / max(1, args.steps + args.warmup)))
    rows = int(max(1, min(n, step_budget / per_row)))
    times = []
    for i in range(args.warmup + args.steps):
        r0 = (i * rows) % max(1, n - rows)
        t0 = time.perf_counter()
        orc.join(wl.R[r0:r0 + rows], wl.R, wl.eps, oracle.MODE_RXS)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    pairs = rows * n
    value = pairs * len(times) / sum(times) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "self_clustered_262k", "n": n, "d": wl.d, "eps": wl.eps,
                   "step_sample": f"{rows} rows x {n} rows"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{rows} query rows x all {n} rows per step, FP64 nested loop, 1 thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1812_07607_gb300 import build as B
    B.build()
    from paper_1812_07607_gb300 import dl

    wl = load_workload(rank)
    n, d = wl.R.shape
    P = wl.pairs
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    feats = torch.from_numpy(wl.R).to(dev)
    ids = torch.from_numpy(wl.r_ids).to(dev)
    store = dl.Store(ids, feats)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as tdist
            tdist.barrier()
        torch.cuda.synchronize()

    def one_step(timing=True):
        res = dl.sim_join(store, None, wl.eps, precision=args.precision, stream=stream, timing=timing)
        st = res.stats()
        res.free()
        return st

    for _ in range(5):   # setup: the tile autotuner's trial calls for this shape class (4 candidates + 1)
        one_step()
    for _ in range(args.warmup):
        one_step()
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    launches0 = dl.kernel_launches()
    step_ms, main_ms, stats = [], [], None
    barrier()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats = one_step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        main_ms.append(stats["ms_main"])
    barrier()
    launches = dl.kernel_launches() - launches0
    clocks = sampler.stop()
    value, total_ms = aggregate(sum(step_ms), P, args.steps, ws, dev)
    ms_per_step = total_ms / args.steps

    # ---- end to end through the C ABI from pinned host memory (store upload + join + pair download)
    h_feats = torch.from_numpy(wl.R).pin_memory()
    h_ids = torch.from_numpy(wl.r_ids).pin_memory()
    e2e_ms = []
    d2h = 0
    for i in range(2 + max(3, args.steps // 4)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = dl.Store(h_ids, h_feats, stream=stream)
        res = dl.sim_join(s2, None, wl.eps, precision=args.precision, stream=stream)
        r_ids, s_ids = res.pairs_host(copy=False)   # the pairs in pinned host memory
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) * 1e3
        d2h = r_ids.nbytes + s_ids.nbytes + 32
        res.free()
        s2.close()
        if i >= 2:
            e2e_ms.append(dt)
    e2e_value = P / (statistics.median(e2e_ms) / 1e3) / 1e9
    h2d = h_feats.numel() * 4 + h_ids.numel() * 8

    # ---- plain FP32 SIMT join on the same GPU (the comparison baseline; not exact)
    plain = None
    if not args.no_baselines:
        one = lambda: dl.sim_join(store, None, wl.eps, precision="fp32_plain", stream=stream, timing=True)
        r = one()
        r.free()
        pm = []
        for _ in range(3):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = one()
            e1.record(stream)
            e1.synchronize()
            pm.append(e0.elapsed_time(e1))
            r.free()
        plain = {"value": P / (statistics.median(pm) / 1e3) / 1e9, "unit": UNIT,
                 "ms_per_step": statistics.median(pm), "kernel": "k8_simt_join (FP32 FMA, inexact at eps)"}

    pk = peaks()
    flops = 2.0 * d * P
    kern_ms = statistics.median(main_ms)
    achieved = flops / (kern_ms / 1e3) / 1e12
    roof = {"bound": "tensor", "achieved": achieved, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
            "frac": achieved / pk["bf16_tflops"], "traffic": traffic_record(),
            "kernel": "tc_join_kernel<256>", "kernel_ms": kern_ms,
            "peak_kind": f"bf16 dense burst ({pk['source']})",
            "algorithmic": f"2*d flops/pair x {P} pairs = {flops:.4g} flops per launch"}

    latency = None
    if rank == 0 and not args.no_latency:
        latency = latency_leg(dl)
    batch = None
    if rank == 0 and not args.no_batch:
        batch = batch_leg(dl)
    serving = None
    if rank == 0 and not args.no_serving:
        serving = serving_leg(dl, seconds=args.serving_seconds, rates=(args.serving_rate, 1000.0, 500.0))
    precision = None
    if rank == 0 and not args.no_precision:
        precision = precision_leg(dl)
    rows = None
    if rank == 0 and not args.no_rows:
        try:
            rows = rows_leg(dl, clocks.get("sm_mhz"))
        except Exception as exc:   # a failing further row must not cost the bench line
            rows = {"error": repr(exc)[:300]}

    cpu = None
    if rank == 0 and not args.no_baselines:
        v1, info1 = cpu_oracle_rate(wl, args.cpu_seconds)
        single = {"value": v1, "unit": UNIT, "cores": 1,
                  "sample": f"{info1['rows']} query rows x all {n} rows ({info1['pairs']} pairs, "
                            f"{info1['seconds']} s), FP64 nested loop, 1 thread"}
        try:
            va, infoa = cpu_oracle_all_cores(wl, info1["seconds"] / info1["rows"], args.cpu_seconds)
            cpu = {"value": va, "unit": UNIT, "cores": infoa["cores"], "kind": "oracle",
                   "cpu_model": infoa["cpu_model"],
                   "sample": f"{infoa['rows']} query rows x all {n} rows ({infoa['pairs']} pairs) in "
                             f"{infoa['seconds']} s: the single-threaded FP64 nested loop in {infoa['cores']} "
                             f"spawned processes, one row shard each",
                   "single_core": single}
        except Exception as exc:   # the single-core figure still stands
            cpu = dict(single, kind="oracle", all_cores_error=repr(exc)[:200])
        try:
            cpu["configs"] = cpu_oracle_configs()
        except Exception as exc:
            cpu["configs"] = {"error": repr(exc)[:200]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "self_clustered_262k", "n": n, "d": d, "eps": wl.eps, "pairs_per_step": P,
                       "mode": "self-join, unordered pairs", "precision": args.precision,
                       "pairs_out": stats["pairs_out"], "band_pairs": stats["band_pairs"],
                       "fp64_pairs": stats["fp64_pairs"], "tile_n": stats["tile_n"],
                       "l2": "512 MiB memset between timed steps (outside the events)",
                       "parallelism": f"replicas x{ws}"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "ms_per_step": statistics.median(e2e_ms)},
            "gpu_launches": int(launches),
            "roofline": roof,
            "cpu_baseline": cpu,
            "plain_fp32_gpu": plain,
            "latency_2k": latency,
            "batch": batch,
            "serving": serving,
            "precision": precision,
            "next_rows": rows,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    store.close()
    if ws > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()
    return 0


def _case_fp8_unit_d512():
    """65,536 x 65,536 d=512 unit-norm R x S join in FP8 e4m3 (the precision config's rows at a
    size that a full ncu capture handles)."""
    import torch
    from paper_1812_07607_gb300 import dl, workloads as W
    dl.load()
    g = W.rng(5)
    R, c = W.unit_mixture(g, 65536, 512, 4096, 0.02)
    T, _ = W.unit_mixture(g, 65536, 512, 4096, 0.02, centroids=c)
    Rs = dl.Store(torch.arange(65536).cuda(), torch.from_numpy(R).cuda())
    Ts = dl.Store(torch.arange(65536).cuda(), torch.from_numpy(T).cuda())
    return lambda: dl.sim_join(Rs, Ts, 0.55, precision="fp8", timing=True)


def _case_pair_unit_d512(pair: int = 2, prec: str = "bf16"):
    """The same 65,536 x 65,536 d=512 join in BF16 with the tensor-core pass on SM pairs
    (cta_group::2, 256-row tiles), or with pair=1 on one SM per tile."""
    import torch
    from paper_1812_07607_gb300 import dl, workloads as W
    dl.load()
    g = W.rng(5)
    R, c = W.unit_mixture(g, 65536, 512, 4096, 0.02)
    T, _ = W.unit_mixture(g, 65536, 512, 4096, 0.02, centroids=c)
    Rs = dl.Store(torch.arange(65536).cuda(), torch.from_numpy(R).cuda())
    Ts = dl.Store(torch.arange(65536).cuda(), torch.from_numpy(T).cuda())
    return lambda: dl.sim_join(Rs, Ts, 0.55, precision=prec, cta_pair=pair, tile_n=256, timing=True)


def _case_serve_batch_258():
    """One serving-sized batch: 258 requests of the serving mix (70% eps at selectivity
    U[0.05%, 0.5%], 30% top-k with k in {1, 10, 100}, sizes lognormal(4, 1.5) in [1, 4096]) in
    one dl_batch_join against the 4,194,304 x 256 serving store, queries on the device."""
    import torch
    from paper_1812_07607_gb300 import dl, workloads as W
    dl.load()
    sw = W.serve_store_4m()
    g = W.rng(SEED_SERVE + 77)
    reqs = W.request_mix(g, 258, 4.0, 1.5, 4096, topk_frac=0.3, ks=(1, 10, 100), sel_lo=5e-4, sel_hi=5e-3)
    table = sw.eps_table()
    off = 0
    for r in reqs:
        r["q_begin"] = off
        off += r["nq"]
        if r["kind"] == "eps":
            r["eps"] = W.eps_for_selectivity(table, r["selectivity"])
    Q = sw.queries(off, SEED_SERVE + 78)
    store = dl.Store(torch.from_numpy(sw.ids).cuda(), torch.from_numpy(sw.X).cuda())
    Qd = torch.from_numpy(Q).cuda()
    qd = torch.arange(off, dtype=torch.int64).cuda()
    return lambda: dl.batch_join(store, qd, Qd, reqs, timing=True)


def _case_batch_decide_1m_d256():
    """64 epsilon requests of 256 fresh queries each at 0.3% selectivity in one dl_batch_join
    against a 1,048,576-row d=256 store drawn like the serving store (32 rows per centre): a
    band-heavy decision pass (k_batch_decide) at a size a full ncu capture handles."""
    import torch
    from paper_1812_07607_gb300 import dl, workloads as W
    dl.load()
    X, _ = W.clustered_histograms(W.rng(SEED_SERVE + 90), 1 << 20, 256, 32768, 0.01)
    Q = W.clustered_queries(64 * 256, SEED_SERVE + 91, SEED_SERVE + 90, 256, 32768, 0.01)
    eps = W.eps_for_selectivity(W.eps_table()["serve_store_4m:selectivity_eps"], 3e-3)
    reqs = [{"kind": "eps", "q_begin": 256 * i, "nq": 256, "eps": eps} for i in range(64)]
    store = dl.Store(torch.arange(X.shape[0]).cuda(), torch.from_numpy(X).cuda())
    Qd = torch.from_numpy(Q).cuda()
    qd = torch.arange(Q.shape[0], dtype=torch.int64).cuda()
    return lambda: dl.batch_join(store, qd, Qd, reqs, timing=True)


def _case_topk_1m_d256(k: int = 100, warps: int = 8):
    """4,096 fresh queries x a 1,048,576-row d=256 clustered store, top-k, the given epilogue."""
    import torch
    from paper_1812_07607_gb300 import dl, workloads as W
    dl.load()
    X, _ = W.clustered_histograms(W.rng(77), 1 << 20, 256, 32768, 0.01)
    Q = W.clustered_queries(4096, 78, 77, 256, 32768, 0.01)
    S = dl.Store(torch.arange(X.shape[0]).cuda(), torch.from_numpy(X).cuda())
    Qs = dl.Store(torch.arange(Q.shape[0]).cuda(), torch.from_numpy(Q).cuda())
    return lambda: dl.topk_join(Qs, S, k, precision="bf16", tile_n=256, epilogue_warps=warps, timing=True)


def _case_dense_d256():
    """16,384 fresh queries x the first 1,048,576 rows of the serving store (d=256), eps at
    0.5% selectivity: a candidate-dense join (BF16, tile 256)."""
    import torch
    from paper_1812_07607_gb300 import dl, workloads as W
    dl.load()
    sw = W.serve_store_4m(n=1048576)
    Q = sw.queries(16384, 7)
    S = dl.Store(torch.from_numpy(sw.ids).cuda(), torch.from_numpy(sw.X).cuda())
    Qs = dl.Store(torch.arange(16384).cuda(), torch.from_numpy(Q).cuda())
    eps = W.eps_for_selectivity(W.eps_table()["serve_store_4m:selectivity_eps"], 5e-3)
    return lambda: dl.sim_join(Qs, S, eps, precision="bf16", timing=True, tile_n=256)


def _case_color_hist_1080p():
    """The colour-histogram transformer on the full traffic_boxes_1080p workload (400 MB of frames)."""
    import torch
    from paper_1812_07607_gb300 import dl, workloads as W
    dl.load()
    wl = W.traffic_boxes_1080p()
    fr = torch.from_numpy(wl.frames).cuda()
    bx = torch.from_numpy(wl.boxes).cuda()
    out = torch.empty((len(wl.boxes), 128), dtype=torch.float32, device="cuda")
    return lambda: dl.color_hist(fr, bx, wl.bins, out=out)


def _case_l1_16k():
    """L1 self-join of the first 16,384 rows of hist_clustered_64k (CUDA-core kernel k8_simt_join<1>)."""
    import torch
    from paper_1812_07607_gb300 import dl, workloads as W
    dl.load()
    X, thr = W.hist_clustered_64k()
    Xs = dl.Store(torch.arange(16384).cuda(), torch.from_numpy(X[:16384]).cuda())
    return lambda: dl.sim_join(Xs, None, thr["l1"], metric="l1", timing=True)


def _case_pruned_tracked():
    """The pruned self-join of tracked_objects_262k on its clustered store (1,024 centres, 5 iterations)."""
    import torch
    from paper_1812_07607_gb300 import dl, workloads as W
    dl.load()
    wt = W.tracked_objects_262k()
    St = dl.Store(torch.from_numpy(wt.r_ids).cuda(), torch.from_numpy(wt.R).cuda())
    Ct = St.clustered(1024, iters=5)
    return lambda: dl.sim_join(Ct, None, wt.eps, precision="bf16", timing=True, prune=True)


PROFILE_CASES = {"fp8_unit_d512_65536": _case_fp8_unit_d512, "dense_d256_16384x1m": _case_dense_d256,
                 "pair_bf16_d512_65536": _case_pair_unit_d512,
                 "serve_batch_258": _case_serve_batch_258,
                 "batch_decide_1m_d256": _case_batch_decide_1m_d256,
                 "topk100_1m_d256_w8": lambda: _case_topk_1m_d256(100, 8),
                 "topk100_1m_d256_w16": lambda: _case_topk_1m_d256(100, 16),
                 "topk10_1m_d256_w8": lambda: _case_topk_1m_d256(10, 8),
                 "topk10_1m_d256_w16": lambda: _case_topk_1m_d256(10, 16),
                 "single_bf16_d512_65536": lambda: _case_pair_unit_d512(pair=1),
                 "pruned_tracked_262k": _case_pruned_tracked,
                 "color_hist_1080p": _case_color_hist_1080p, "l1_hist_16384": _case_l1_16k}


def run_profile_case(name, calls=3):
    from paper_1812_07607_gb300 import build as B
    B.build()
    call = PROFILE_CASES[name]()
    import torch
    for _ in range(calls):
        t0 = time.perf_counter()
        r = call()
        torch.cuda.synchronize()
        dt = 1e3 * (time.perf_counter() - t0)
        if not hasattr(r, "stats"):
            print(json.dumps({"case": name, "ms_call": dt}), flush=True)
            continue
        st = r.stats()
        r.free()
        print(json.dumps({"case": name, "ms_call": dt, "ms_main": st["ms_main"], "ms_recheck": st["ms_recheck"],
                          "band_pairs": st["band_pairs"], "pairs_out": st["pairs_out"], "tile_n": st.get("tile_n"),
                          "epilogue_warps": st.get("epilogue_warps")}), flush=True)
    return 0


def main():
    args = parse()
    if args.profile_case:
        return run_profile_case(args.profile_case, args.profile_calls)
    if args.peak_probe:
        print(json.dumps(peak_probe()), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
