"""Batching and serving at full size, checked against the oracle on sampled requests.

  * Batching: 4,096 eps / top-k (k = 10) requests in ONE dl_batch_join call against the
    2,097,152 x 128 store; sizes lognormal(5, 1.5) in [1, 8192]; eps at a selectivity
    uniform in [0.05%, 0.5%] of the store. 64 seeded requests are checked, up to four
    seeded query rows each, against the oracle over the whole store.
  * Serving: the request loop over the 4,194,304 x 256 store with Poisson arrivals
    (2,000 requests/s; 70% eps at the same selectivities, 30% top-k with k in
    {1, 10, 100}, sizes lognormal(4, 1.5) in [1, 4096]); 32 seeded requests are checked
    against the oracle on sampled rows, and six of them against the same request run
    alone through the single-request calls (same result alone and in the mix).
"""

import time

import numpy as np
import pytest

from oracle_pool import OraclePool
from paper_1812_07607_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dl():
    import torch
    from paper_1812_07607_gb300 import build as B, dl as D
    assert torch.cuda.is_available()
    B.build()
    D.load()
    return D


def _requests(store, n_req, mu, sigma, qmax, ks, seed):
    g = W.rng(seed)
    reqs = W.request_mix(g, n_req, mu, sigma, qmax, topk_frac=0.3, ks=ks, sel_lo=5e-4, sel_hi=5e-3)
    table = store.eps_table()
    off = 0
    for r in reqs:
        r["q_begin"] = off
        off += r["nq"]
        if r["kind"] == "eps":
            r["eps"] = W.eps_for_selectivity(table, r["selectivity"])
    return reqs, off


def _sample_rows(g, nq, m):
    return np.sort(g.choice(nq, size=min(m, nq), replace=False))


def test_batch_2m_store_4096_requests_sampled(dl):
    import torch
    st = W.batch_store_2m()
    reqs, nq_total = _requests(st, 4096, 5.0, 1.5, 8192, (10,), W.SEED_BASE + 74)
    Q = st.queries(nq_total, W.SEED_BASE + 75)
    qid = np.arange(nq_total, dtype=np.int64) * 5 + 3
    g = W.rng(W.SEED_BASE + 76)
    picks = np.sort(g.choice([i for i, r in enumerate(reqs) if r["nq"] > 0], size=64, replace=False))
    with OraclePool(st.X) as op:
        jobs_e, jobs_k = [], []
        for i in picks.tolist():
            r = reqs[i]
            rows = _sample_rows(g, r["nq"], 4) + r["q_begin"]
            for q in rows.tolist():
                (jobs_e if r["kind"] == "eps" else jobs_k).append((i, q))
        want_e = op.within([Q[q] for _, q in jobs_e], [reqs[i]["eps"] ** 2 for i, _ in jobs_e])
        want_k = op.topk([Q[q] for _, q in jobs_k], [reqs[i]["k"] for i, _ in jobs_k])
        store = dl.Store(torch.from_numpy(st.ids).cuda(), torch.from_numpy(st.X).cuda())
        res = dl.batch_join(store, torch.from_numpy(qid).cuda(), torch.from_numpy(Q).cuda(), reqs)
        stats = res.stats()
        assert stats["pairs_evaluated"] == nq_total * st.X.shape[0]
        rows_of = {}
        for i, q in jobs_e:
            rows_of.setdefault(i, []).append(q)
        got_e, got_k = {}, {}
        for i in picks.tolist():
            if reqs[i]["kind"] == "eps":
                a, b = res.request_pairs(i)
                order = np.argsort(a, kind="stable")   # group the request's pairs by query row
                a, b = a[order], b[order]
                for q in rows_of.get(i, []):
                    lo, hi = np.searchsorted(a, qid[q], "left"), np.searchsorted(a, qid[q], "right")
                    got_e[(i, q)] = np.sort(b[lo:hi])
            else:
                got_k[i] = res.request_topk(i)
        res.free()
        for (i, q), idx in zip(jobs_e, want_e.get()):
            got = got_e[(i, q)]
            assert np.unique(got).shape[0] == got.shape[0]   # no duplicate pairs
            assert np.array_equal(got, np.sort(st.ids[idx])), (i, q, got.shape, idx.shape)
        for (i, q), (idx, d2) in zip(jobs_k, want_k.get()):
            ids, dd = got_k[i]
            row = q - reqs[i]["q_begin"]
            assert np.array_equal(ids[row], st.ids[idx]) and np.array_equal(dd[row], d2), (i, q)
    assert len(jobs_e) > 50 and len(jobs_k) > 20
    assert stats["pairs_out"] > 10**9


def test_serving_4m_store_poisson_sampled(dl):
    import torch
    sv_wl = W.serve_store_4m()
    reqs, nq_total = _requests(sv_wl, 600, 4.0, 1.5, 4096, (1, 10, 100), W.SEED_BASE + 84)
    Q = sv_wl.queries(nq_total, W.SEED_BASE + 85)
    g = W.rng(W.SEED_BASE + 86)
    arrivals = np.cumsum(g.exponential(1.0 / 2000.0, size=len(reqs)))
    picks = set(np.sort(g.choice([i for i, r in enumerate(reqs) if r["nq"] > 0], size=32, replace=False)).tolist())
    alone = sorted(picks)[:6]
    with OraclePool(sv_wl.X) as op:
        jobs_e, jobs_k = [], []
        for i in sorted(picks):
            r = reqs[i]
            for q in (_sample_rows(g, r["nq"], 2) + r["q_begin"]).tolist():
                (jobs_e if r["kind"] == "eps" else jobs_k).append((i, q))
        want_e = op.within([Q[q] for _, q in jobs_e], [reqs[i]["eps"] ** 2 for i, _ in jobs_e])
        want_k = op.topk([Q[q] for _, q in jobs_k], [reqs[i]["k"] for i, _ in jobs_k])
        store = dl.Store(torch.from_numpy(sv_wl.ids).cuda(), torch.from_numpy(sv_wl.X).cuda())
        server = dl.Server(store, mem_budget_bytes=64 << 30, slots=3, max_batch_rows=65536)
        tickets = []
        t0 = time.perf_counter()
        for i, r in enumerate(reqs):
            while time.perf_counter() - t0 < arrivals[i]:
                pass
            q0, nq = r["q_begin"], r["nq"]
            qid = np.arange(q0, q0 + nq, dtype=np.int64)
            if r["kind"] == "eps":
                tickets.append(server.submit(qid, Q[q0:q0 + nq], "eps", eps=r["eps"]))
            else:
                tickets.append(server.submit(qid, Q[q0:q0 + nq], "topk", k=r["k"]))
        kept = {}
        for i, t in enumerate(tickets):
            res = None
            for _ in range(1200):
                res = server.poll(t, timeout_us=100_000)
                if res is not None:
                    break
            assert res is not None, f"request {i} did not finish"
            if i in picks:
                kept[i] = res.pairs_host() if reqs[i]["kind"] == "eps" else res.topk_host()
            res.free()
        sstats = server.stats()
        server.close()
        for (i, q), idx in zip(jobs_e, want_e.get()):
            a, b = kept[i]
            assert np.array_equal(np.sort(b[a == q]), np.sort(sv_wl.ids[idx])), (i, q)
        for (i, q), (idx, d2) in zip(jobs_k, want_k.get()):
            ids, dd = kept[i]
            row = q - reqs[i]["q_begin"]
            assert np.array_equal(ids[row], sv_wl.ids[idx]) and np.array_equal(dd[row], d2), (i, q)
        for i in alone:   # the same request alone, through the single-request calls
            r = reqs[i]
            q0, nq = r["q_begin"], r["nq"]
            Qs = dl.Store(torch.arange(q0, q0 + nq).cuda(), torch.from_numpy(Q[q0:q0 + nq]).cuda())
            if r["kind"] == "eps":
                one = dl.sim_join(Qs, store, r["eps"])
                a, b = one.pairs_host()
                ka, kb = kept[i]
                assert set(zip(a.tolist(), b.tolist())) == set(zip(ka.tolist(), kb.tolist())), i
            else:
                one = dl.topk_join(Qs, store, r["k"])
                ids, dd = one.topk_host()
                assert np.array_equal(ids, kept[i][0]) and np.array_equal(dd, kept[i][1]), i
            one.free()
    assert sstats["completed"] == len(reqs) and sstats["failed"] == 0
    assert sstats["p99_ms"] >= sstats["p50_ms"] > 0
