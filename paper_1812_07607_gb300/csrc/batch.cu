// batch.cu -- many epsilon-join and top-k requests of uneven sizes in one call.
//
// The paper's image-matching queries (Sec. 6.2, q1 near-duplicates and q4
// deduplication) are issued here many at a time against one resident store.
// Every epsilon-join row of every request goes into ONE persistent tensor-core
// launch: the per-row thresholds (k_rowpar) carry each row's own eps, so tiles
// may mix requests freely. Every top-k row goes into one top-k launch with the
// largest k as heap size and each row's own k in the finalize. Outputs are then
// routed to their requests:
//   k_batch_expand   request table -> per query row: caller row, eps^2 or k,
//                    request index and output slot;
//   tc_join_kernel   candidates (proven matches and band pairs) of all eps rows;
//   k_batch_decide   settles band pairs exactly and counts each request's pairs;
//   k_batch_scatter  writes every request's id pairs into its own segment.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "checked.cuh"
#include "exact.cuh"
#include "kernels.h"

namespace dl {

struct ReqDev {
    int64_t q_begin;   // first caller row
    int64_t seg_off;   // first expanded row
    int64_t out_off;   // top-k: first output slot
    double e2;         // eps^2 (eps requests)
    int32_t k;         // top-k requests
    int32_t req;       // index in the caller's request table
};

__global__ void k_batch_expand(const ReqDev *__restrict__ reqs, int n, int64_t total, int32_t *__restrict__ gather,
                               double *__restrict__ row_e2, float2 *__restrict__ row_t, int d, int *__restrict__ row_k,
                               int64_t *__restrict__ row_off, int32_t *__restrict__ row_req)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    int lo = 0, hi = n - 1;
    while (lo < hi) {   // last request whose segment starts at or before i
        const int mid = (lo + hi + 1) >> 1;
        if (reqs[mid].seg_off <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    const ReqDev r = reqs[lo];
    const int64_t local = i - r.seg_off;
    gather[i] = (int32_t)(r.q_begin + local);
    if (row_e2) row_e2[i] = r.e2;
    if (row_t) {   // the row's FP32 thresholds of the exact decision
        float ta, tr;
        fp32_thresholds(r.e2, d, &ta, &tr);
        row_t[i] = make_float2(ta, tr);
    }
    if (row_k) row_k[i] = r.k;
    if (row_off) row_off[i] = r.out_off + local * r.k;
    row_req[i] = r.req;
}

// Candidates -> decisions in place (rejected entries get column 0xffffffff) and
// per-request counts. One thread per entry; the warp rechecks its band entries
// together (FP32 with its bound, then the float-float sum, canonical FP64 if neither
// decides); counts are aggregated per warp over lanes of the same request.
__global__ void __launch_bounds__(256)
    k_batch_decide(uint2 *__restrict__ cand, const unsigned long long *__restrict__ cand_cnt, unsigned long long cap,
                   const float *__restrict__ Q, const float *__restrict__ S, int d, const double *__restrict__ row_e2,
                   const float2 *__restrict__ row_t, const int32_t *__restrict__ row_req,
                   unsigned long long *__restrict__ req_cnt,
                   unsigned long long *__restrict__ n_fp64, unsigned long long *__restrict__ n_band, int nQ, int nS)
{
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long n = min(*cand_cnt, cap);
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x;
    uint2 nxt = base + threadIdx.x < n ? cand[base + threadIdx.x] : make_uint2(0u, 0u);
    for (; base < n; base += stride) {
        const unsigned long long i = base + threadIdx.x;   // warp-uniform loop bound: base < n
        bool valid = i < n;
        const uint2 e = nxt;
        // the next window's entry loads while this one is decided (no entry is read after its write)
        nxt = i + stride < n ? cand[i + stride] : make_uint2(0u, 0u);
        if (valid && !DL_CHECK(e.x < (unsigned)nQ && (e.y & ~kBandFlag) < (unsigned)nS, 30, i)) {
            cand[i] = make_uint2(0u, 0xffffffffu);   // checked build: dropped, so the scatter skips it
            valid = false;
        }
        const int r = (int)e.x;
        const int c = (int)(e.y & ~kBandFlag);
        const bool band = valid && (e.y & kBandFlag);
        bool acc = valid && !band;
        bool f64 = false;
        const unsigned bm = __ballot_sync(0xffffffffu, band);
        if (bm) {
            double e2 = 0.0;
            float ta = 0.f, tr = 0.f;
            if (band) {   // the row's thresholds, computed once per row at expansion
                e2 = row_e2[r];
                const float2 t2 = row_t[r];
                ta = t2.x;
                tr = t2.y;
            }
            const bool dec = warp_band_decide(bm, Q + (size_t)r * d, S + (size_t)c * d, d, e2, ta, tr, &f64);
            if (band) acc = dec;
        }
        const unsigned fm = __ballot_sync(0xffffffffu, f64);
        if (lane == 0) {
            if (bm) atomicAdd(n_band, (unsigned long long)__popc(bm));
            if (fm) atomicAdd(n_fp64, (unsigned long long)__popc(fm));
        }
        grouped_add(req_cnt, acc ? row_req[r] : 0, acc, 1u);
        if (valid) cand[i] = acc ? make_uint2((uint32_t)r, (uint32_t)c) : make_uint2((uint32_t)r, 0xffffffffu);
    }
}

__global__ void __launch_bounds__(256)
    k_batch_scatter(const uint2 *__restrict__ cand, const unsigned long long *__restrict__ cand_cnt,
                    unsigned long long cap, const int32_t *__restrict__ row_req, const int64_t *__restrict__ req_off,
                    unsigned long long *__restrict__ cursor, const int64_t *__restrict__ q_ids,
                    const int64_t *__restrict__ s_ids, int64_t *__restrict__ out_r, int64_t *__restrict__ out_s)
{
    const unsigned long long n = min(*cand_cnt, cap);
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x;
    uint2 nxt = base + threadIdx.x < n ? cand[base + threadIdx.x] : make_uint2(0u, 0xffffffffu);
    for (; base < n; base += stride) {
        const unsigned long long i = base + threadIdx.x;
        const bool valid = i < n;
        const uint2 e = nxt;
        nxt = i + stride < n ? cand[i + stride] : make_uint2(0u, 0xffffffffu);   // the next window, early
        const bool acc = valid && e.y != 0xffffffffu;
        const int32_t q = acc ? row_req[e.x] : 0;
        const unsigned long long pos = grouped_add(cursor, q, acc, 1u);
        if (acc) {
            const int64_t o = req_off[q] + (int64_t)pos;
            out_r[o] = q_ids[e.x];
            out_s[o] = s_ids[e.y];
        }
    }
}

static size_t al(size_t x) { return (x + 255) & ~size_t(255); }

// Units of the epsilon pass: every row tile against every S tile (no self pairs), in
// S-range-major order so that the CTAs running together share S tiles through L2.
static int batch_units(int64_t nR, int64_t nS, int BN, int sms, std::vector<int4> *v)
{
    const int mt = (int)((nR + 127) / 128), nt = (int)((nS + BN - 1) / BN);
    int L = 64;
    while (L > 1 && (int64_t)mt * ((nt + L - 1) / L) < 4LL * sms) L >>= 1;
    v->clear();
    for (int nb = 0; nb < nt; nb += L)
        for (int m = 0; m < mt; ++m) v->push_back(make_int4(m, nb, std::min(nb + L, nt), 0));
    return DL_OK;
}

}  // namespace dl

using namespace dl;

extern "C" int dl_batch_join(const dl_store *S, const int64_t *q_ids, const float *q_feats, int64_t nq_total,
                             int32_t d, int32_t where, const dl_request *reqs, int32_t n_req, const dl_join_opts *opts,
                             dl_result **out)
{
    dl::NvtxScope nvtx_scope("dl_batch_join");
    clear_error();
    if (!out) {
        set_error("dl_batch_join: out is NULL");
        return DL_EINVAL;
    }
    *out = nullptr;
    if (!S || !reqs || n_req < 1 || nq_total < 0 || (nq_total > 0 && (!q_ids || !q_feats))) {
        set_error("dl_batch_join: bad arguments");
        return DL_EINVAL;
    }
    if (d != S->d) {
        set_error("dl_batch_join: dimension mismatch %d vs %d", d, S->d);
        return DL_EINVAL;
    }
    if (where != DL_MEM_HOST && where != DL_MEM_DEVICE) {
        set_error("dl_batch_join: bad memory kind");
        return DL_EINVAL;
    }
    dl_join_opts o;
    if (opts)
        o = *opts;
    else
        dl_join_opts_default(&o);
    cudaStream_t st = (cudaStream_t)o.cuda_stream;
    int dev = -1;
    DL_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != S->device) {
        set_error("dl_batch_join: store lives on another device");
        return DL_EINVAL;
    }
    // ---- request tables (host bookkeeping of n_req entries)
    std::vector<ReqDev> er, kr;
    int64_t ne = 0, nk = 0, slots = 0;
    std::vector<int64_t> topk_off(n_req + 1, 0);
    for (int i = 0; i < n_req; ++i) {
        const dl_request &q = reqs[i];
        if (q.nq < 0 || q.q_begin < 0 || q.q_begin + q.nq > nq_total) {
            set_error("dl_batch_join: request %d rows out of range", i);
            return DL_EINVAL;
        }
        ReqDev r{};
        r.q_begin = q.q_begin;
        r.req = i;
        if (q.kind == DL_REQ_EPS) {
            if (std::isnan(q.eps) || q.eps < 0.0) {
                set_error("dl_batch_join: request %d has eps %g", i, q.eps);
                return DL_EINVAL;
            }
            r.seg_off = ne;
            r.e2 = q.eps * q.eps;
            r.k = 0;
            ne += q.nq;
            er.push_back(r);
        } else if (q.kind == DL_REQ_TOPK) {
            if (q.k < 1 || q.k > 1024) {
                set_error("dl_batch_join: request %d has k=%d", i, q.k);
                return DL_EINVAL;
            }
            r.seg_off = nk;
            r.k = q.k;
            r.out_off = slots;
            topk_off[i] = slots;
            slots += q.nq * q.k;
            nk += q.nq;
            kr.push_back(r);
        } else {
            set_error("dl_batch_join: request %d has kind %d", i, q.kind);
            return DL_EINVAL;
        }
    }
    // top-k rows are grouped by k (each group runs with its own heap size)
    std::stable_sort(kr.begin(), kr.end(), [](const ReqDev &a, const ReqDev &b) { return a.k < b.k; });
    std::vector<std::pair<int, std::pair<int64_t, int64_t>>> kgroups;   // k -> [first row, end row)
    {
        int64_t off = 0;
        for (auto &r : kr) {
            const int64_t nq = reqs[r.req].nq;
            r.seg_off = off;
            if (kgroups.empty() || kgroups.back().first != r.k) kgroups.push_back({r.k, {off, off}});
            off += nq;
            kgroups.back().second.second = off;
        }
    }
    if (ne >= (int64_t(1) << 31) || nk >= (int64_t(1) << 31)) {
        set_error("dl_batch_join: too many query rows");
        return DL_EINVAL;
    }
    const int sms = device_sm_count();
    int rc = DL_OK;
    std::vector<void *> frees;
    std::vector<dl_store *> stores;
    // opts.timing: events at [0] start, [1]/[2] around the epsilon contraction, [3] after the
    // exact decisions, [4] after the scatter, [5] end (after the top-k part)
    cudaEvent_t bev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    if (o.timing)
        for (auto &ev : bev) cudaEventCreate(&ev);
    auto mark = [&](int i) {
        if (bev[i]) cudaEventRecord(bev[i], st);
    };
    auto cleanup = [&]() {
        cudaStreamSynchronize(st);   // nothing of this call may still run when its scratch is released
        for (auto *s : stores) dl_store_destroy(s);
        for (void *p : frees) dev_free(p, st);
        cudaStreamSynchronize(st);
        for (auto &ev : bev)
            if (ev) {
                cudaEventDestroy(ev);
                ev = nullptr;
            }
    };
    mark(0);
    // ---- query rows on the device (host inputs are uploaded once)
    const int64_t *dq_ids = q_ids;
    const float *dq = q_feats;
    if (where == DL_MEM_HOST && nq_total > 0) {
        void *up = nullptr;
        rc = dev_alloc(&up, al(nq_total * 8) + al(nq_total * (size_t)d * 4), st);
        if (rc) return rc;
        frees.push_back(up);
        cudaError_t e = cudaMemcpyAsync(up, q_ids, nq_total * 8, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync((char *)up + al(nq_total * 8), q_feats, nq_total * (size_t)d * 4,
                                cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            cleanup();
            return cuda_fail(e, "dl_batch_join upload");
        }
        dq_ids = (const int64_t *)up;
        dq = (const float *)((char *)up + al(nq_total * 8));
    }
    // ---- expansion: per-row parameters of both parts
    const size_t b_tab = al((er.size() + kr.size()) * sizeof(ReqDev));
    const size_t b_e = al(ne * 4) + al(ne * 8) + al(ne * 4) + al(ne * 8);
    const size_t b_k = al(nk * 4) + al(nk * 4) + al(nk * 8) + al(nk * 4);
    void *meta = nullptr;
    rc = dev_alloc(&meta, b_tab + b_e + b_k + 256, st);
    if (rc) {
        cleanup();
        return rc;
    }
    frees.push_back(meta);
    char *pm = (char *)meta;
    ReqDev *d_er = (ReqDev *)pm, *d_kr = d_er + er.size();
    pm += b_tab;
    int32_t *g_e = (int32_t *)pm;
    pm += al(ne * 4);
    double *row_e2 = (double *)pm;
    pm += al(ne * 8);
    int32_t *req_e = (int32_t *)pm;
    pm += al(ne * 4);
    float2 *row_t = (float2 *)pm;
    pm += al(ne * 8);
    int32_t *g_k = (int32_t *)pm;
    pm += al(nk * 4);
    int *row_k = (int *)pm;
    pm += al(nk * 4);
    int64_t *row_off = (int64_t *)pm;
    pm += al(nk * 8);
    int32_t *req_k = (int32_t *)pm;
    std::vector<ReqDev> tab(er);
    tab.insert(tab.end(), kr.begin(), kr.end());
    if (!tab.empty()) {
        cudaError_t e = cudaMemcpyAsync(d_er, tab.data(), tab.size() * sizeof(ReqDev), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            cleanup();
            return cuda_fail(e, "dl_batch_join request table");
        }
    }
    if (ne > 0) {
        k_batch_expand<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(d_er, (int)er.size(), ne, g_e, row_e2, row_t, d,
                                                                      nullptr, nullptr, req_e);
        count_launch();
    }
    if (nk > 0) {
        k_batch_expand<<<(unsigned)((nk + 255) / 256), 256, 0, st>>>(d_kr, (int)kr.size(), nk, g_k, nullptr, nullptr, d,
                                                                      row_k, row_off, req_k);
        count_launch();
    }
    // ---- result block: eps pairs are sized after the count pass; top-k slots now
    std::vector<int64_t> pair_off(n_req + 1, 0);
    int64_t total_pairs = 0;
    dl_join_stats stats{};
    stats.precision = DL_PREC_BF16;
    void *tk_block = nullptr;
    if (slots > 0) {
        rc = dev_alloc(&tk_block, al(slots * 8) * 2, st);
        if (rc) {
            cleanup();
            return rc;
        }
    }
    void *pair_block = nullptr;
    // ---- epsilon part
    if (ne > 0 && S->n > 0) {
        dl_store *Qe = nullptr;
        rc = store_create_impl(&Qe, dq_ids, dq, ne, d, DL_MEM_DEVICE, st, g_e);
        if (rc) {
            dev_free(tk_block, st);
            cleanup();
            return rc;
        }
        stores.push_back(Qe);
        if (Qe->dp > 512) {
            dev_free(tk_block, st);
            cleanup();
            set_error("dl_batch_join: epsilon requests need d <= 512 (d=%d)", d);
            return DL_EUNSUPPORTED;
        }
        bool tune_trial = false;
        const int code = o.tile_n ? o.tile_n : tune_pick(Qe->dp, kTuneBatch, ne, S->n, &tune_trial);
        const int BN = tune_bn(code);
        const bool wide = tune_wide(code);
        stats.tile_n = BN;   // the epsilon rows' configuration (the autotuner's choice once decided)
        stats.cta_pair = 1;
        stats.epilogue_warps = wide ? 16 : 8;
        const int64_t mt = (ne + 127) / 128;
        cudaEvent_t tev[2] = {nullptr, nullptr};
        if (tune_trial)
            for (auto &ev : tev) cudaEventCreate(&ev);
        std::vector<int4> units;
        batch_units(ne, S->n, BN, sms, &units);
        int64_t cap;
        {
            std::lock_guard<std::mutex> lk(const_cast<dl_store *>(S)->mu);
            // candidates per evaluated pair from the last batch against this store, with headroom
            const double want = S->hint_batch_rate * (double)ne * (double)S->n;
            cap = std::max<int64_t>(1 << 20, (int64_t)(want * 1.3) + (1 << 16));
        }
        for (int attempt = 0;; ++attempt) {
            void *ws = nullptr;
            const size_t b_units = al(units.size() * sizeof(int4)), b_rowpar = al(mt * 128 * sizeof(float4)),
                         b_cand = al(cap * sizeof(uint2)), b_rc = al((size_t)n_req * 8) * 3;
            rc = dev_alloc(&ws, 256 + b_units + b_rowpar + b_cand + b_rc, st);
            if (rc) break;
            char *pw = (char *)ws;
            unsigned long long *cnt = (unsigned long long *)pw;   // [0] cand [1] fp64 [2] band [3] err
            pw += 256;
            int4 *d_units = (int4 *)pw;
            pw += b_units;
            float4 *rowpar = (float4 *)pw;
            pw += b_rowpar;
            uint2 *cand = (uint2 *)pw;
            pw += b_cand;
            unsigned long long *req_cnt = (unsigned long long *)pw;
            int64_t *req_off = (int64_t *)(pw + al((size_t)n_req * 8));
            unsigned long long *cursor = (unsigned long long *)(pw + 2 * al((size_t)n_req * 8));
            cudaError_t e = cudaMemsetAsync(ws, 0, 256, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(req_cnt, 0, (size_t)n_req * 8, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, (size_t)n_req * 8, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(d_units, units.data(), units.size() * sizeof(int4), cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "dl_batch_join eps setup");
                dev_free(ws, st);
                break;
            }
            rc = launch_rowpar(Qe->nq64, Qe->rowb, ne, mt * 128, Qe->dp, 0.0, row_e2, gamma64(d), rowpar, st);
            const CUtensorMap *tmA = nullptr, *tmB = nullptr;
            if (!rc) rc = get_tmap(Qe, 128, &tmA);
            if (!rc) rc = get_tmap(const_cast<dl_store *>(S), BN, &tmB);
            if (!rc) {
                TcLaunch L;
                std::memset(&L.p, 0, sizeof L.p);
                L.tmA = tmA;
                L.tmB = tmB;
                L.BN = BN;
                L.grid = std::min((int)units.size(), sms);
                L.p.units = d_units;
                L.p.n_units = (int)units.size();
                L.p.nR = (int)ne;
                L.p.nS = (int)S->n;
                L.p.kc = Qe->dp / 64;
                tc_plan(BN, Qe->dp / 64, &L.p.stages, &L.p.a_slots, false, false, wide, true);
                L.wide = wide;
                L.p.upper = 0;
                L.p.rowpar = rowpar;
                L.p.beta = S->beta;
                L.p.cstat = S->cstat;
                L.p.cand = cand;
                L.p.cand_cnt = cnt + 0;
                L.p.cand_cap = (unsigned long long)cap;
                L.p.err = (int *)(cnt + 3);
                if (tune_trial) cudaEventRecord(tev[0], st);
                mark(1);
                rc = launch_tc_join(L, st);
                mark(2);
                if (tune_trial) cudaEventRecord(tev[1], st);
            }
            if (!rc) {
                k_batch_decide<<<sms * 8, 256, 0, st>>>(cand, cnt + 0, (unsigned long long)cap, Qe->x32, S->x32, d,
                                                        row_e2, row_t, req_e, req_cnt, cnt + 1, cnt + 2, (int)ne,
                                                        (int)S->n);
                count_launch(2);
                e = cudaGetLastError();
                if (e != cudaSuccess) rc = cuda_fail(e, "k_batch_decide launch");
                mark(3);
            }
            unsigned long long hc[4] = {0, 0, 0, 0};
            std::vector<unsigned long long> hreq(n_req, 0);
            if (!rc) {
                e = cudaMemcpyAsync(hc, cnt, sizeof hc, cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaMemcpyAsync(hreq.data(), req_cnt, (size_t)n_req * 8, cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                if (e != cudaSuccess) rc = cuda_fail(e, "dl_batch_join eps");
            }
            if (!rc && hc[3]) {
                set_error("dl_batch_join: a bounded device wait expired");
                rc = DL_ETIMEOUT;
            }
            if (!rc && hc[0] > (unsigned long long)cap) {   // candidate list too small: exact size, re-run
                dev_free(ws, st);
                if (attempt >= 3) {
                    rc = DL_ENOMEM;
                    set_error("dl_batch_join: candidate list keeps overflowing");
                    break;
                }
                cap = (int64_t)hc[0] + (int64_t)(hc[0] / 8) + 1024;
                stats.reruns++;
                continue;
            }
            if (!rc) {
                for (int i = 0; i < n_req; ++i) pair_off[i + 1] = pair_off[i] + (int64_t)hreq[i];
                total_pairs = pair_off[n_req];
                stats.band_pairs = (int64_t)hc[2];
                stats.fp64_pairs = (int64_t)hc[1];
                rc = dev_alloc(&pair_block, al(std::max<int64_t>(total_pairs, 1) * 8) * 2, st);
            }
            if (!rc) {
                e = cudaMemcpyAsync(req_off, pair_off.data(), (size_t)n_req * 8, cudaMemcpyHostToDevice, st);
                if (e != cudaSuccess) rc = cuda_fail(e, "dl_batch_join offsets");
            }
            if (!rc && total_pairs > 0) {
                int64_t *o_r = (int64_t *)pair_block;
                int64_t *o_s = (int64_t *)((char *)pair_block + al(total_pairs * 8));
                k_batch_scatter<<<sms * 8, 256, 0, st>>>(cand, cnt + 0, (unsigned long long)cap, req_e, req_off, cursor,
                                                         Qe->ids, S->ids, o_r, o_s);
                count_launch();
                e = cudaGetLastError();
                if (e != cudaSuccess) rc = cuda_fail(e, "k_batch_scatter launch");
            }
            mark(4);
            if (!rc) {
                std::lock_guard<std::mutex> lk(const_cast<dl_store *>(S)->mu);
                const_cast<dl_store *>(S)->hint_batch_rate = (double)hc[0] / ((double)ne * (double)S->n);
            }
            if (!rc && tune_trial && attempt == 0) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, tev[0], tev[1]);
                tune_record(Qe->dp, kTuneBatch, ne, S->n, code, ms, (double)ne * (double)S->n);
            }
            dev_free(ws, st);
            break;
        }
        for (auto &ev : tev)
            if (ev) cudaEventDestroy(ev);
        if (rc) {
            dev_free(tk_block, st);
            dev_free(pair_block, st);
            cleanup();
            return rc;
        }
    }
    // ---- top-k part
    for (const auto &grp : kgroups) {
        const int kg = grp.first;
        const int64_t g0 = grp.second.first, g1 = grp.second.second;
        if (g1 <= g0) continue;
        dl_store *Qk = nullptr;
        rc = store_create_impl(&Qk, dq_ids, dq, g1 - g0, d, DL_MEM_DEVICE, st, g_k + g0);
        if (!rc) {
            stores.push_back(Qk);
            dl_join_stats ts{};
            rc = topk_core(Qk, S, kg, row_k + g0, row_off + g0, (int64_t *)tk_block,
                           (double *)((char *)tk_block + al(slots * 8)), o, st, &ts);
            stats.fp64_pairs += ts.fp64_pairs;
        }
        if (rc) {
            dev_free(tk_block, st);
            dev_free(pair_block, st);
            cleanup();
            return rc;
        }
    }
    mark(5);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        dev_free(tk_block, st);
        dev_free(pair_block, st);
        cleanup();
        return cuda_fail(e, "dl_batch_join");
    }
    if (o.timing) {
        auto span = [&](int a, int b) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, bev[a], bev[b]) != cudaSuccess) {
                cudaGetLastError();   // an event that was never recorded (that part did not run)
                ms = 0.f;
            }
            return ms;
        };
        stats.ms_main = span(1, 2);
        stats.ms_recheck = span(2, 4);
        stats.ms_total = span(0, 5);
    }
    cleanup();
    dl_result *res = new dl_result();
    res->kind = 2;
    res->device = dev;
    res->stream = st;
    res->count = total_pairs;
    res->cap = total_pairs;
    res->d_r = pair_block ? (int64_t *)pair_block : nullptr;
    res->d_s = pair_block ? (int64_t *)((char *)pair_block + al(std::max<int64_t>(total_pairs, 1) * 8)) : nullptr;
    res->d_ids = tk_block ? (int64_t *)tk_block : nullptr;
    res->d_d2 = tk_block ? (double *)((char *)tk_block + al(slots * 8)) : nullptr;
    res->n_topk_slots = slots;
    res->req_kind.resize(n_req);
    res->req_k.resize(n_req);
    res->req_nq.resize(n_req);
    for (int i = 0; i < n_req; ++i) {
        res->req_kind[i] = reqs[i].kind;
        res->req_k[i] = reqs[i].kind == DL_REQ_TOPK ? reqs[i].k : 0;
        res->req_nq[i] = reqs[i].nq;
    }
    res->pair_off = pair_off;
    res->topk_off = topk_off;
    stats.pairs_out = total_pairs;
    for (int i = 0; i < n_req; ++i)
        stats.pairs_evaluated += reqs[i].nq * S->n;
    res->stats = stats;
    *out = res;
    return DL_OK;
}

DL_CHECK_READER(batch)
