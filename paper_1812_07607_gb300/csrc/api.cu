// api.cu -- the C ABI: join orchestration, results and options.
//
// dl_sim_join runs, on the caller's stream:
//   k_rowpar (per-row thresholds for this eps)           [tensor-core path]
//   tc_join_kernel  or  k8_simt_join                       (classify every pair)
//   k6_recheck (settle the band pairs exactly)             [exact paths]
//   k_diag (self-join full mode: the diagonal)
// then reads the three counters back (one 32-byte copy), re-runs with larger
// buffers if an internal buffer overflowed, and hands the id pairs over as a
// result that stays on the device until the caller asks for a host copy.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "checked.cuh"
#include "kernels.h"

namespace dl {

// ------------------------------------------------------------------ pinned host memory
static thread_local unsigned long long *t_counters = nullptr;

static int pinned_counters(unsigned long long **p)
{
    if (!t_counters) {
        cudaError_t e = cudaHostAlloc((void **)&t_counters, 64, cudaHostAllocDefault);
        if (e != cudaSuccess) {
            t_counters = nullptr;
            return cuda_fail(e, "cudaHostAlloc(counters)");
        }
    }
    *p = t_counters;
    return DL_OK;
}

// A small pool of pinned host blocks, reused across results (pinning is slow).
static std::mutex g_hpool_mu;
static std::multimap<size_t, void *> g_hpool;

static void *hpool_get(size_t bytes, size_t *got)
{
    {
        std::lock_guard<std::mutex> lk(g_hpool_mu);
        auto it = g_hpool.lower_bound(bytes);
        if (it != g_hpool.end() && it->first <= 2 * bytes + (1 << 20)) {
            void *p = it->second;
            *got = it->first;
            g_hpool.erase(it);
            return p;
        }
    }
    void *p = nullptr;
    if (cudaHostAlloc(&p, bytes, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    *got = bytes;
    return p;
}

static void hpool_put(void *p, size_t bytes)
{
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_hpool_mu);
    g_hpool.emplace(bytes, p);
}

// ------------------------------------------------------------------ unit lists
// Work units of the tensor-core kernel: (R tile m, S tiles [nb, ne)). For a
// self-join only tiles holding some column c > row r are listed. Units are ordered
// S-range-major (all R tiles of one range of L S tiles, then the next range), and the
// kernel hands them out round-robin, so the CTAs running at the same time share the
// same S tiles: each S range is read from HBM about once per wave and served from L2
// to every CTA, while each CTA reads only its own R tile. (R-major order would stream
// a different S range into every CTA, which makes a store larger than L2 HBM-bound.)
static std::mutex g_units_mu;
static std::map<std::tuple<int, int64_t, int64_t, int, int, int>, std::pair<int4 *, int>> g_units;

// R tiles are `tr` rows high: 128 for one SM per tile, 256 for an SM pair (which holds
// 128 rows each).
static int first_upper_tile(int m, int BN, bool upper, int tr)
{
    if (!upper) return 0;
    const long long num = (long long)m * tr + 2 - BN;
    return num <= 0 ? 0 : (int)((num + BN - 1) / BN);
}

static void build_units(int64_t nR, int64_t nS, bool upper, int BN, int L, int tr, std::vector<int4> *v)
{
    const int mt = (int)((nR + tr - 1) / tr), nt = (int)((nS + BN - 1) / BN);
    v->clear();
    for (int nb0 = 0; nb0 < nt; nb0 += L)
        for (int m = 0; m < mt; ++m) {
            const int lo = std::max(nb0, first_upper_tile(m, BN, upper, tr)), hi = std::min(nb0 + L, nt);
            if (lo < hi) v->push_back(make_int4(m, lo, hi, 0));
        }
}

static int get_units(int64_t nR, int64_t nS, bool upper, int BN, int sms, const int4 **d_units, int *n_units,
                     int tr = 128)
{
    int dev = 0;
    cudaGetDevice(&dev);
    const int mt = (int)((nR + tr - 1) / tr), nt = (int)((nS + BN - 1) / BN);
    const int workers = (tr == 256) ? sms / 2 : sms;   // SMs, or SM pairs
    // the longest ranges (fewest R re-reads) that still give every worker four units
    int L = 64;
    while (L > 1) {
        long long cnt = 0;
        for (int nb0 = 0; nb0 < nt; nb0 += L)
            for (int m = 0; m < mt; ++m)
                if (std::max(nb0, first_upper_tile(m, BN, upper, tr)) < std::min(nb0 + L, nt)) ++cnt;
        if (cnt >= 4LL * workers) break;
        L >>= 1;
    }
    auto key = std::make_tuple(dev, nR, nS, (int)upper * 1000 + tr, BN, L);
    std::lock_guard<std::mutex> lk(g_units_mu);
    auto it = g_units.find(key);
    if (it == g_units.end()) {
        std::vector<int4> v;
        build_units(nR, nS, upper, BN, L, tr, &v);
        int4 *d = nullptr;
        if (!v.empty()) {
            cudaError_t e = cudaMalloc(&d, v.size() * sizeof(int4));
            if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(units)");
            e = cudaMemcpy(d, v.data(), v.size() * sizeof(int4), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(units)");
        }
        it = g_units.emplace(key, std::make_pair(d, (int)v.size())).first;
    }
    *d_units = it->second.first;
    *n_units = it->second.second;
    return DL_OK;
}

// ------------------------------------------------------------------ one pass of a join
struct PassCfg {
    const dl_store *R, *S;
    bool self, mirror;
    int prec;
    int BN;
    bool cg2 = false;       // tensor-core pass on SM pairs (256-row tiles)
    bool wide = false;      // 16 epilogue warps
    double e2;              // squared-L2 threshold (metric 0), or the L1 / chi-square threshold eps
    int metric;             // 0 squared L2 (and cosine), 1 L1, 2 chi-square
    const int64_t *ids;     // ids written for both sides (self-join only; NULL: the store's ids)
    const int4 *units = nullptr;   // work units of the pruned join
    int n_units = 0;               // (pruned: an upper bound; the count itself is on the device)
    const int *n_units_dev = nullptr;
    const uint32_t *tile_mask = nullptr;   // pruned: tiles of a unit with a clear bit are skipped
    int mask_ntw = 0;
    bool pruned = false;           // the pruned join (units may be empty: every tile pair skipped)
    bool ip = false;               // inner-product join: e2 holds the threshold t of q.x >= t
    float t_acc, t_rej;     // FP32 thresholds (exact: recheck/SIMT; plain: SIMT only)
    int64_t cap, band_cap;
    bool timing;
    cudaStream_t st;
};

struct PassOut {
    int64_t *out_r = nullptr, *out_s = nullptr;
    unsigned long long out_cnt = 0, band_cnt = 0, band_only = 0, fp64_cnt = 0;
    int err = 0;
    float ms_main = 0, ms_recheck = 0, ms_total = 0;
    int launches = 0;
    int grid = 0;           // CTAs of the tensor-core launch
};

static int run_pass(const PassCfg &c, PassOut *po)
{
    const dl_store *R = c.R, *S = c.S;
    cudaStream_t st = c.st;
    const int64_t nR = R->n, nS = S->n;
    const int d = R->d;
    const int sms = device_sm_count();

    // output block (kept by the result) and workspace block (freed here)
    void *outb = nullptr, *ws = nullptr;
    const size_t cap = (size_t)std::max<int64_t>(c.cap, 1);
    int rc = dev_alloc(&outb, 2 * cap * sizeof(int64_t), st);
    if (rc) return rc;
    const int64_t rows_pad = (nR + 255) / 256 * 256;   // per-row parameters cover whole 128- or 256-row tiles
    const size_t b_band = ((size_t)std::max<int64_t>(c.band_cap, 1) * sizeof(uint2) + 255) & ~size_t(255);
    const size_t b_rowpar = (size_t)rows_pad * sizeof(float4);
    rc = dev_alloc(&ws, 256 + b_band + b_rowpar, st);
    if (rc) {
        dev_free(outb, st);
        return rc;
    }
    po->out_r = (int64_t *)outb;
    po->out_s = po->out_r + cap;
    unsigned long long *cnt = (unsigned long long *)ws;   // [0] out [1] band/candidates [2] band pairs [3] fp64 [4] err
    uint2 *band = (uint2 *)((char *)ws + 256);
    float4 *rowpar = (float4 *)((char *)ws + 256 + b_band);

    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    auto cleanup_ws = [&]() {
        dev_free(ws, st);
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    };
    if (c.timing)
        for (auto &e : ev) cudaEventCreate(&e);
    cudaError_t e = cudaMemsetAsync(cnt, 0, 64, st);
    if (e != cudaSuccess) {
        cleanup_ws();
        dev_free(outb, st);
        return cuda_fail(e, "cudaMemsetAsync(counters)");
    }
    if (c.timing) cudaEventRecord(ev[0], st);

    JoinOut jo;
    jo.r_ids = c.ids ? c.ids : R->ids;
    jo.s_ids = c.ids ? c.ids : S->ids;
    jo.out_r = po->out_r;
    jo.out_s = po->out_s;
    jo.out_cnt = cnt + 0;
    jo.out_cap = (unsigned long long)c.cap;
    jo.band = band;
    jo.band_cnt = cnt + 1;
    jo.band_cap = (unsigned long long)c.band_cap;
    jo.mirror = c.mirror ? 1 : 0;
    jo.orig = (c.self && !c.mirror) ? R->orig : nullptr;

    int launches = 0;
    if (nR > 0 && nS > 0) {
        NvtxScope nvtx_pass("join pass: distances, bounds, compaction, recheck");
        if (c.prec == DL_PREC_BF16 || c.prec == DL_PREC_FP8E4M3) {
            const bool fp8 = c.prec == DL_PREC_FP8E4M3;
            if (fp8) {
                rc = ensure_fp8(const_cast<dl_store *>(R), st);
                if (!rc) rc = ensure_fp8(const_cast<dl_store *>(S), st);
            }
            if (!rc && c.ip) rc = ensure_ip(const_cast<dl_store *>(S), st);
            if (!rc && c.ip)
                rc = launch_rowpar_ip(R->rowb, nR, rows_pad, R->dp, c.e2, rowpar, st);
            else if (!rc)
                rc = launch_rowpar(R->nq64, R->rowb, nR, rows_pad, R->dp, c.e2, nullptr, gamma64(d), rowpar, st,
                                   fp8 ? R->rowb8 : nullptr);
            ++launches;
            const CUtensorMap *tmA = nullptr, *tmB = nullptr;
            if (!rc) rc = fp8 ? get_tmap8(const_cast<dl_store *>(R), 128, &tmA) : get_tmap(const_cast<dl_store *>(R), 128, &tmA);
            const int b_rows = c.cg2 ? c.BN / 2 : c.BN;   // an SM pair loads half of each S tile per SM
            if (!rc)
                rc = fp8 ? get_tmap8(const_cast<dl_store *>(S), b_rows, &tmB) : get_tmap(const_cast<dl_store *>(S), b_rows, &tmB);
            const int4 *units = nullptr;
            int n_units = 0;
            if (!rc && c.units) {
                units = c.units;
                n_units = c.n_units;
            } else if (!rc && !c.pruned) {
                rc = get_units(nR, nS, c.self, c.BN, sms, &units, &n_units, c.cg2 ? 256 : 128);
            }
            if (!rc && n_units > 0) {
                TcLaunch L;
                std::memset(&L.p, 0, sizeof L.p);
                L.tmA = tmA;
                L.tmB = tmB;
                L.BN = c.BN;
                L.cg2 = c.cg2;
                L.wide = c.wide;
                L.grid = c.cg2 ? 2 * std::min(n_units, sms / 2) : std::min(n_units, sms);
                L.p.units = units;
                L.p.n_units = n_units;
                L.p.n_units_dev = c.n_units_dev;
                L.p.tile_mask = c.tile_mask;
                L.p.mask_ntw = c.mask_ntw;
                L.p.nR = (int)nR;
                L.p.nS = (int)nS;
                L.p.kc = fp8 ? R->dp8 / 128 : R->dp / 64;
                tc_plan(c.BN, L.p.kc, &L.p.stages, &L.p.a_slots, fp8, c.cg2, c.wide, !c.pruned);
                L.p.upper = c.self ? 1 : 0;
                L.p.rowpar = rowpar;
                L.p.beta = c.ip ? S->beta_ip : S->beta;
                L.p.cstat = fp8 ? S->cstat8 : (c.ip ? S->cstat_ip : S->cstat);
                L.p.sc_r = fp8 ? R->sc8 : nullptr;
                L.p.sc_s = fp8 ? S->scc8 : nullptr;
                L.p.cand = band;                 // candidates share the band buffer and counter
                L.p.cand_cnt = cnt + 1;
                L.p.cand_cap = (unsigned long long)c.band_cap;
                L.p.err = (int *)(cnt + 4);
                rc = launch_tc_join(L, st, false, fp8, &po->grid);
                ++launches;
            }
        } else {
            SimtParams sp{};
            sp.R = R->x32;
            sp.S = S->x32;
            sp.nR = (int)nR;
            sp.nS = (int)nS;
            sp.d = d;
            sp.upper = c.self ? 1 : 0;
            sp.tiles_m = 0;
            sp.exact = (c.prec == DL_PREC_FP32) ? 1 : 0;
            sp.metric = c.metric;
            sp.t_acc = c.t_acc;
            sp.t_rej = c.t_rej;
            sp.out = jo;
            rc = launch_simt_join(sp, st);
            ++launches;
        }
        if (c.timing) cudaEventRecord(ev[1], st);
        nvtxRangePushA("exact recheck of the band (K6)");
        if (!rc && c.ip) {
            rc = launch_finalize_ip(band, cnt + 1, (unsigned long long)c.band_cap, R->x32, S->x32, d, c.e2, jo, cnt + 3,
                                    cnt + 2, sms * 8, st, (int)nR, (int)nS);
            ++launches;
        } else if (!rc && (c.prec == DL_PREC_BF16 || c.prec == DL_PREC_FP8E4M3)) {
            rc = launch_finalize(band, cnt + 1, (unsigned long long)c.band_cap, R->x32, S->x32, d, c.e2, c.t_acc,
                                 c.t_rej, jo, cnt + 3, cnt + 2, sms * 8, st, (int)nR, (int)nS);
            ++launches;
        } else if (!rc && c.prec == DL_PREC_FP32 && c.metric != 0) {
            rc = launch_hist_recheck(c.metric, band, cnt + 1, (unsigned long long)c.band_cap, R->x32, S->x32, d, c.e2,
                                     jo, cnt + 3, sms * 8, st);
            ++launches;
        } else if (!rc && c.prec == DL_PREC_FP32) {
            rc = launch_recheck(band, cnt + 1, (unsigned long long)c.band_cap, R->x32, S->x32, d, c.e2, c.t_acc, c.t_rej,
                                jo, cnt + 3, sms * 8, st);
            ++launches;
        }
        nvtxRangePop();
        if (c.timing) cudaEventRecord(ev[2], st);
    } else if (c.timing) {
        cudaEventRecord(ev[1], st);
        cudaEventRecord(ev[2], st);
    }
    if (!rc && c.mirror) {
        rc = launch_diag(c.ids ? c.ids : R->ids, nR, po->out_r, po->out_s, cnt + 0, (unsigned long long)c.cap, st);
        ++launches;
    }
    if (c.timing) cudaEventRecord(ev[3], st);
    unsigned long long *hc = nullptr;
    if (!rc) rc = pinned_counters(&hc);
    if (!rc) {
        e = cudaMemcpyAsync(hc, cnt, 40, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "join kernels");
    }
    if (!rc) {
        po->out_cnt = hc[0];
        po->band_cnt = hc[1];                                  // list fill (band or candidate list)
        po->band_only = (c.prec == DL_PREC_BF16 || c.prec == DL_PREC_FP8E4M3) ? hc[2] : hc[1];
        po->fp64_cnt = hc[3];
        po->err = (int)hc[4];
        if (c.timing) {
            cudaEventElapsedTime(&po->ms_main, ev[0], ev[1]);
            cudaEventElapsedTime(&po->ms_recheck, ev[1], ev[2]);
            cudaEventElapsedTime(&po->ms_total, ev[0], ev[3]);
        }
    }
    po->launches = launches;
    cleanup_ws();
    if (rc) {
        dev_free(outb, st);
        po->out_r = po->out_s = nullptr;
    }
    return rc;
}

// Output and band pairs per evaluated pair of the last completed join (any store): the first
// join of a new store sizes its buffers from them.
static std::mutex g_rate_mu;
static double g_rate_out = 0.0, g_rate_band = 0.0;

static int check_device(const dl_store *s)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != s->device) {
        set_error("store lives on device %d but device %d is current", s->device, dev);
        return DL_EINVAL;
    }
    return DL_OK;
}

}  // namespace dl

using namespace dl;

extern "C" {

void dl_join_opts_default(dl_join_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->precision = DL_PREC_AUTO;
    o->self_mode = DL_SELF_UPPER;
}

}  // extern "C"

namespace dl {

int sim_join_impl(const dl_store *R, const dl_store *S, int32_t metric, double eps, const dl_join_opts *opts,
                  dl_result **out, const int64_t *emit_ids)
{
    if (!out) {
        set_error("dl_sim_join: out is NULL");
        return DL_EINVAL;
    }
    *out = nullptr;
    if (!R) {
        set_error("dl_sim_join: R is NULL");
        return DL_EINVAL;
    }
    double e2 = 0.0;   // the squared-L2 threshold the join decides against
    if (metric == DL_METRIC_L2) {
        if (std::isnan(eps) || eps < 0.0) {
            set_error("dl_sim_join: eps must be >= 0 (got %g)", eps);
            return DL_EINVAL;
        }
        e2 = eps * eps;
    } else if (metric == DL_METRIC_COSINE) {
        // eps is the cosine threshold c: on unit-normalized rows cos >= c is D <= 2 - 2c
        if (!(eps >= -1.0 && eps <= 1.0)) {
            set_error("dl_sim_join: the cosine threshold must lie in [-1, 1] (got %g)", eps);
            return DL_EINVAL;
        }
        if (!R->unit || (S && !S->unit)) {
            set_error("dl_sim_join: the cosine metric needs stores made by dl_store_normalize");
            return DL_EINVAL;
        }
        e2 = 2.0 - 2.0 * eps;
    } else if (metric == DL_METRIC_L1 || metric == DL_METRIC_CHI2) {
        if (std::isnan(eps) || eps < 0.0) {
            set_error("dl_sim_join: eps must be >= 0 (got %g)", eps);
            return DL_EINVAL;
        }
        e2 = eps;   // histogram distances are compared unsquared
    } else if (metric == DL_METRIC_IP) {
        if (std::isnan(eps)) {
            set_error("dl_sim_join: the inner-product threshold is NaN");
            return DL_EINVAL;
        }
        e2 = eps;   // the threshold t of q.x >= t
    } else {
        set_error("dl_sim_join: unsupported metric %d", metric);
        return DL_EINVAL;
    }
    const int hmetric = (metric == DL_METRIC_L1) ? 1 : (metric == DL_METRIC_CHI2) ? 2 : 0;
    dl_join_opts o;
    if (opts)
        o = *opts;
    else
        dl_join_opts_default(&o);
    const bool self = (S == nullptr);
    const dl_store *Sx = self ? R : S;
    if (Sx->d != R->d) {
        set_error("dl_sim_join: dimension mismatch %d vs %d", R->d, Sx->d);
        return DL_EINVAL;
    }
    if (o.self_mode != DL_SELF_UPPER && o.self_mode != DL_SELF_FULL) {
        set_error("dl_sim_join: bad self_mode %d", o.self_mode);
        return DL_EINVAL;
    }
    int rc = check_device(R);
    if (!rc) rc = check_device(Sx);
    if (rc) return rc;
    int prec = o.precision;
    // AUTO: BF16 while its R tile fits in shared memory (d <= 512), else the FP8 tensor-core
    // path (d <= 1024, always within the domain); both give the exact set. The histogram
    // distances are not contractions: they run on the CUDA cores (FP32 + bound + FP64).
    const bool ip = metric == DL_METRIC_IP;
    if (prec == DL_PREC_AUTO)
        prec = hmetric ? DL_PREC_FP32 : (ip || R->dp <= 512) ? DL_PREC_BF16 : DL_PREC_FP8E4M3;
    if (ip && (prec != DL_PREC_BF16 || (self && o.self_mode == DL_SELF_FULL) || o.prune)) {
        set_error("dl_sim_join: the inner-product join runs in BF16, R x S or the upper self mode, without pruning");
        return DL_EUNSUPPORTED;
    }
    if (hmetric && (prec == DL_PREC_BF16 || prec == DL_PREC_FP8E4M3)) {
        set_error("dl_sim_join: L1 and chi-square run on DL_PREC_FP32 (or FP32_PLAIN), not on tensor cores");
        return DL_EUNSUPPORTED;
    }
    if (hmetric == 2) {
        bool ok = false;
        rc = store_nonneg(const_cast<dl_store *>(R), (cudaStream_t)o.cuda_stream, &ok);
        if (!rc && ok && !self) rc = store_nonneg(const_cast<dl_store *>(Sx), (cudaStream_t)o.cuda_stream, &ok);
        if (rc) return rc;
        if (!ok) {
            set_error("dl_sim_join: the chi-square distance needs non-negative features");
            return DL_EINVAL;
        }
    }
    if (prec != DL_PREC_BF16 && prec != DL_PREC_FP8E4M3 && prec != DL_PREC_FP32 && prec != DL_PREC_FP32_PLAIN) {
        set_error("dl_sim_join: bad precision %d", prec);
        return DL_EINVAL;
    }
    if (prec == DL_PREC_BF16 && R->dp > 512) {
        set_error("dl_sim_join: BF16 tensor-core path supports d <= 512 (d=%d)", R->d);
        return DL_EUNSUPPORTED;
    }
    if (o.tile_n != 0 && o.tile_n != 128 && o.tile_n != 256) {
        set_error("dl_sim_join: tile_n must be 0, 128 or 256");
        return DL_EINVAL;
    }
    if (o.cta_pair < 0 || o.cta_pair > 2 || (o.cta_pair == 2 && (o.tile_n == 128 || o.prune))) {
        set_error("dl_sim_join: cta_pair must be 0, 1 or 2 (2: tile_n 0 or 256, no prune)");
        return DL_EINVAL;
    }
    if ((o.epilogue_warps != 0 && o.epilogue_warps != 8 && o.epilogue_warps != 16) ||
        (o.epilogue_warps == 16 && (o.tile_n == 128 || o.cta_pair == 2))) {
        set_error("dl_sim_join: epilogue_warps must be 0, 8 or 16 (16: tile_n 0 or 256, one SM per tile)");
        return DL_EINVAL;
    }
    // tile configuration: given, or autotuned per shape class (tensor-core precisions, dense join)
    const bool tc = prec == DL_PREC_BF16 || prec == DL_PREC_FP8E4M3;
    const int tune_kind = (prec == DL_PREC_FP8E4M3) ? (self ? kTuneEpsSelf8 : kTuneEpsRxS8)
                                                    : (self ? kTuneEpsSelf : kTuneEpsRxS);
    bool tune_trial = false;
    int code = (o.tile_n ? o.tile_n : 256) | (o.cta_pair == 2 ? kTunePair : 0) | (o.epilogue_warps == 16 ? kTuneWide : 0);
    if (tc && !o.prune && o.tile_n == 0 && o.cta_pair == 0 && o.epilogue_warps == 0)
        code = tune_pick(R->dp, tune_kind, R->n, Sx->n, &tune_trial);
    const int BN = tune_bn(code);
    const bool cg2 = tc && tune_pair(code);
    const bool wide = tc && tune_wide(code);
    if (prec == DL_PREC_FP8E4M3 && R->d > 1024) {
        set_error("dl_sim_join: FP8 path supports d <= 1024");
        return DL_EUNSUPPORTED;
    }
    if (o.out_capacity < 0) {
        set_error("dl_sim_join: negative out_capacity");
        return DL_EINVAL;
    }

    const int d = R->d;
    PassCfg c;
    c.R = R;
    c.S = Sx;
    c.self = self;
    c.mirror = self && o.self_mode == DL_SELF_FULL;
    c.prec = prec;
    c.BN = BN;
    c.cg2 = cg2;
    c.wide = wide;
    c.e2 = e2;
    c.metric = hmetric;
    c.ip = ip;
    c.ids = emit_ids;
    if (prec == DL_PREC_FP32_PLAIN && hmetric) {
        c.t_acc = (float)eps;
        c.t_rej = c.t_acc;
    } else if (prec == DL_PREC_FP32_PLAIN) {
        const float ef = (float)std::sqrt(e2);
        c.t_acc = ef * ef;
        c.t_rej = c.t_acc;
    } else if (hmetric) {
        // |D32 - D| <= g32 D + abs32 for the SIMT evaluation, |D64 - D| <= g64 D for the canonical sum
        const double g64 = (hmetric == 1) ? gamma64(d) : gamma64(d + 4);
        const double g32 = (hmetric == 1) ? (d + 4) * 1.1920928955078125e-07 : (d + 16) * 1.1920928955078125e-07;
        const double abs32 = (hmetric == 1) ? d * 7.52316384526264e-37 : d * 2.168404344971009e-19;   // d 2^-120, d 2^-62
        c.t_acc = f32_rd(eps * (1.0 - g64) * (1.0 - g32) * (1.0 - 8.881784197001252e-16) - abs32);
        c.t_rej = f32_ru(eps * (1.0 + 2.0 * g64) * (1.0 + g32) * (1.0 + 8.881784197001252e-16) + abs32);
    } else {
        const double g64 = gamma64(d), g32 = gamma32(d);
        const double abs32 = (double)(d + 8) * 1.401298464324817e-45 * 2.0;
        c.t_acc = f32_rd(e2 * (1.0 - g64) * (1.0 - g32) * (1.0 - 8.881784197001252e-16) - abs32);
        c.t_rej = f32_ru(e2 * (1.0 + 2.0 * g64) * (1.0 + g32) * (1.0 + 8.881784197001252e-16) + abs32);
    }
    c.timing = o.timing != 0 || tune_trial;
    c.st = (cudaStream_t)o.cuda_stream;
    const bool fixed = o.out_capacity > 0;
    const double n_pairs = self ? 0.5 * (double)R->n * (double)R->n : (double)R->n * (double)Sx->n;
    {
        std::lock_guard<std::mutex> lk(const_cast<dl_store *>(R)->mu);
        int64_t hp = R->hint_pairs, hb = R->hint_band;
        if (hp == 0 && hb == 0) {   // a store's first join: the process-wide rates of the last join
            // (a short first call costs a re-run; capped so that an outlier cannot claim GBs)
            std::lock_guard<std::mutex> lr(g_rate_mu);
            hp = (int64_t)std::min(g_rate_out * n_pairs, (double)(1 << 26));
            hb = (int64_t)std::min(g_rate_band * n_pairs, (double)(1 << 26));
        }
        c.cap = fixed ? o.out_capacity : std::max<int64_t>(1 << 16, hp + hp / 4);
        // the BF16 path's candidate list holds proven matches and band pairs
        const int64_t want = ((prec == DL_PREC_BF16 || prec == DL_PREC_FP8E4M3) ? hp : 0) + hb;
        c.band_cap = std::max<int64_t>(1 << 16, want + want / 4);
    }

    PruneUnits pu;
    int64_t tiles_total = 0, tiles_kept = 0;
    if (o.prune && (prec == DL_PREC_BF16 || prec == DL_PREC_FP8E4M3) && hmetric == 0) {
        rc = prune_units(R, Sx, self, BN, e2, c.st, &pu);
        if (rc) return rc;
        c.units = pu.units;
        c.n_units = pu.cap;
        c.n_units_dev = pu.count;
        c.tile_mask = pu.mask;
        c.mask_ntw = pu.ntw;
        c.pruned = true;
        tiles_total = pu.total;
    }
    struct UnitsGuard {
        void *p;
        cudaStream_t st;
        ~UnitsGuard()
        {
            if (p) dev_free(p, st);
        }
    } units_guard{pu.block, c.st};
    PassOut po;
    int reruns = 0;
    for (int attempt = 0;; ++attempt) {
        po = PassOut();
        rc = run_pass(c, &po);
        if (rc) return rc;
        if (po.err) {
            dev_free(po.out_r, c.st);
            set_error("dl_sim_join: a bounded device wait expired (kernel pipeline stalled)");
            return DL_ETIMEOUT;
        }
        const bool band_over = po.band_cnt > (unsigned long long)c.band_cap;   // candidate / band list
        const bool out_over = po.out_cnt > (unsigned long long)c.cap;
        if (band_over || (out_over && !fixed)) {
            if (attempt >= 4) {
                dev_free(po.out_r, c.st);
                set_error("dl_sim_join: output keeps overflowing");
                return DL_ENOMEM;
            }
            dev_free(po.out_r, c.st);
            if (band_over) c.band_cap = (int64_t)po.band_cnt + (int64_t)(po.band_cnt / 8) + 1024;
            if (out_over) c.cap = (int64_t)po.out_cnt + (int64_t)(po.out_cnt / 8) + 1024;
            ++reruns;
            continue;
        }
        break;
    }
    if (pu.kept) {   // the surviving tile pairs (the stream has drained: one small read)
        unsigned long long kept = 0;
        cudaError_t e = cudaMemcpyAsync(&kept, pu.kept, sizeof kept, cudaMemcpyDeviceToHost, c.st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
        if (e != cudaSuccess) {
            dev_free(po.out_r, c.st);
            return cuda_fail(e, "dl_sim_join: pruned tile count");
        }
        tiles_kept = (int64_t)kept;
    }
    {
        std::lock_guard<std::mutex> lk(const_cast<dl_store *>(R)->mu);
        const_cast<dl_store *>(R)->hint_pairs = (int64_t)po.out_cnt;
        const_cast<dl_store *>(R)->hint_band = (int64_t)po.band_only;
    }
    if (n_pairs > 0) {
        std::lock_guard<std::mutex> lr(g_rate_mu);
        g_rate_out = (double)po.out_cnt / n_pairs;
        g_rate_band = (double)po.band_only / n_pairs;
    }
    if (tune_trial && reruns == 0)
        tune_record(R->dp, tune_kind, R->n, Sx->n, code, po.ms_main,
                    self ? 0.5 * (double)R->n * (double)R->n : (double)R->n * (double)Sx->n);
    dl_result *res = new dl_result();
    res->kind = 0;
    res->device = R->device;
    res->stream = c.st;
    res->count = (int64_t)po.out_cnt;
    res->cap = c.cap;
    res->d_r = po.out_r;
    res->d_s = po.out_s;
    dl_join_stats &s = res->stats;
    s.pairs_evaluated = self ? (c.mirror ? R->n * R->n : R->n * (R->n - 1) / 2) : R->n * Sx->n;
    s.pairs_out = (int64_t)po.out_cnt;
    s.band_pairs = (int64_t)po.band_only;
    s.fp64_pairs = (int64_t)po.fp64_cnt;
    s.reruns = reruns;
    s.precision = prec;
    s.tile_n = (prec == DL_PREC_BF16 || prec == DL_PREC_FP8E4M3) ? BN : 0;
    s.cta_pair = (prec == DL_PREC_BF16 || prec == DL_PREC_FP8E4M3) ? (cg2 ? 2 : 1) : 0;
    s.epilogue_warps = (prec == DL_PREC_BF16 || prec == DL_PREC_FP8E4M3) ? (wide ? 16 : 8) : 0;
    s.ms_main = po.ms_main;
    s.ms_recheck = po.ms_recheck;
    s.ms_total = po.ms_total;
    s.kernels_launched = po.launches * (reruns + 1);
    s.grid_ctas = po.grid;
    s.tile_pairs = tiles_total;
    s.tile_pairs_kept = tiles_kept;
    *out = res;
    if (fixed && po.out_cnt > (unsigned long long)c.cap) {
        set_error("dl_sim_join: %llu pairs exceed out_capacity %lld", po.out_cnt, (long long)c.cap);
        return DL_EOVERFLOW;
    }
    return DL_OK;
}

}  // namespace dl

namespace dl {
int check_read_join_tc(unsigned long long *out);
int check_read_topk(unsigned long long *out);
int check_read_recheck(unsigned long long *out);
int check_read_batch(unsigned long long *out);
}  // namespace dl

#ifdef DL_CHECKED
// Records a failed check on a constant-false condition: no memory access is guarded or made.
__global__ void k_check_selftest(long long index) { DL_CHECK(false, 99, index); }
#endif

DL_CHECK_READER(api)

extern "C" {

int dl_sim_join(const dl_store *R, const dl_store *S, int32_t metric, double eps, const dl_join_opts *opts,
                dl_result **out)
{
    dl::NvtxScope nvtx_scope("dl_sim_join");
    clear_error();
    return sim_join_impl(R, S, metric, eps, opts, out, nullptr);
}

int dl_topk_join(const dl_store *Q, const dl_store *S, int32_t metric, int32_t k, const dl_join_opts *opts,
                 dl_result **out);   // defined in topk.cu

int dl_debug_scores(const dl_store *R, const dl_store *S, int32_t precision, float *h_out, float *e_out,
                    void *cuda_stream)
{
    dl::NvtxScope nvtx_scope("dl_debug_scores");
    clear_error();
    if (!R || !S || !h_out || !e_out || R->d != S->d) {
        set_error("dl_debug_scores: bad arguments");
        return DL_EINVAL;
    }
    if (precision != DL_PREC_BF16 && precision != DL_PREC_FP8E4M3) {
        set_error("dl_debug_scores: precision must be BF16 or FP8");
        return DL_EINVAL;
    }
    if (R->n * S->n > (int64_t(1) << 28) || R->n == 0 || S->n == 0) {
        set_error("dl_debug_scores: |R| |S| must be in [1, 2^28]");
        return DL_EINVAL;
    }
    const bool fp8 = precision == DL_PREC_FP8E4M3;
    if ((!fp8 && R->dp > 512) || (fp8 && R->d > 1024)) {
        set_error("dl_debug_scores: d too large for this precision");
        return DL_EUNSUPPORTED;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int rc = DL_OK;
    if (fp8) {
        rc = ensure_fp8(const_cast<dl_store *>(R), st);
        if (!rc) rc = ensure_fp8(const_cast<dl_store *>(S), st);
        if (rc) return rc;
    }
    const int64_t mt = (R->n + 127) / 128;
    void *ws = nullptr;
    rc = dev_alloc(&ws, 256 + mt * 128 * sizeof(float4) + 65536 * sizeof(uint2), st);
    if (rc) return rc;
    unsigned long long *cnt = (unsigned long long *)ws;
    float4 *rowpar = (float4 *)((char *)ws + 256);
    uint2 *cand = (uint2 *)((char *)rowpar + mt * 128 * sizeof(float4));
    cudaMemsetAsync(cnt, 0, 256, st);
    // thresholds for eps = 0 (the dump does not depend on them; candidates are discarded)
    rc = launch_rowpar(R->nq64, R->rowb, R->n, mt * 128, R->dp, 0.0, nullptr, gamma64(R->d), rowpar, st,
                       fp8 ? R->rowb8 : nullptr);
    const CUtensorMap *tmA = nullptr, *tmB = nullptr;
    const int BN = 256;
    if (!rc) rc = fp8 ? get_tmap8(const_cast<dl_store *>(R), 128, &tmA) : get_tmap(const_cast<dl_store *>(R), 128, &tmA);
    if (!rc) rc = fp8 ? get_tmap8(const_cast<dl_store *>(S), BN, &tmB) : get_tmap(const_cast<dl_store *>(S), BN, &tmB);
    const int4 *units = nullptr;
    int n_units = 0;
    if (!rc) rc = get_units(R->n, S->n, false, BN, device_sm_count(), &units, &n_units);
    if (!rc) {
        TcLaunch L;
        std::memset(&L.p, 0, sizeof L.p);
        L.tmA = tmA;
        L.tmB = tmB;
        L.BN = BN;
        L.grid = std::min(n_units, device_sm_count());
        L.p.units = units;
        L.p.n_units = n_units;
        L.p.nR = (int)R->n;
        L.p.nS = (int)S->n;
        L.p.kc = fp8 ? R->dp8 / 128 : R->dp / 64;
        tc_plan(BN, L.p.kc, &L.p.stages, &L.p.a_slots, fp8);
        L.p.rowpar = rowpar;
        L.p.beta = S->beta;
        L.p.cstat = fp8 ? S->cstat8 : S->cstat;
        L.p.sc_r = fp8 ? R->sc8 : nullptr;
        L.p.sc_s = fp8 ? S->scc8 : nullptr;
        L.p.cand = cand;
        L.p.cand_cnt = cnt + 0;
        L.p.cand_cap = 65536;
        L.p.err = (int *)(cnt + 1);
        L.p.dump_h = h_out;
        L.p.dump_e = e_out;
        L.p.orig_r = R->orig;
        L.p.orig_s = S->orig;
        rc = launch_tc_join(L, st, false, fp8);
    }
    cudaError_t e = cudaStreamSynchronize(st);
    dev_free(ws, st);
    if (!rc && e != cudaSuccess) rc = cuda_fail(e, "dl_debug_scores");
    return rc;
}

int dl_result_count(const dl_result *r, int64_t *n)
{
    if (!r || !n) {
        set_error("dl_result_count: NULL argument");
        return DL_EINVAL;
    }
    *n = (r->kind == 0 || r->kind == 2) ? r->count : r->nq * r->k;
    return DL_OK;
}

int dl_result_pairs(dl_result *r, int32_t where, const int64_t **r_ids, const int64_t **s_ids, int64_t *n)
{
    if (!r || r->kind != 0) {
        set_error("dl_result_pairs: not an epsilon-join result");
        return DL_EINVAL;
    }
    const int64_t cnt = std::min(r->count, r->cap);
    if (n) *n = cnt;
    if (where == DL_MEM_DEVICE) {
        if (r_ids) *r_ids = r->d_r;
        if (s_ids) *s_ids = r->d_s;
        return DL_OK;
    }
    if (where != DL_MEM_HOST) {
        set_error("dl_result_pairs: bad memory kind");
        return DL_EINVAL;
    }
    if (!r->h_r) {
        size_t got = 0;
        const size_t bytes = std::max<size_t>(16, (size_t)cnt * 2 * sizeof(int64_t));
        void *h = hpool_get(bytes, &got);
        if (!h) {
            set_error("dl_result_pairs: pinned host allocation of %zu bytes failed", bytes);
            return DL_ENOMEM;
        }
        r->h_r = (int64_t *)h;
        r->h_s = r->h_r + cnt;
        r->h_bytes = got;
        cudaError_t e = cudaSuccess;
        if (cnt > 0) e = cudaMemcpyAsync(r->h_r, r->d_r, cnt * sizeof(int64_t), cudaMemcpyDeviceToHost, r->stream);
        if (e == cudaSuccess && cnt > 0)
            e = cudaMemcpyAsync(r->h_s, r->d_s, cnt * sizeof(int64_t), cudaMemcpyDeviceToHost, r->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
        if (e != cudaSuccess) return cuda_fail(e, "dl_result_pairs copy");
    }
    if (r_ids) *r_ids = r->h_r;
    if (s_ids) *s_ids = r->h_s;
    return DL_OK;
}

int dl_result_topk(dl_result *r, int32_t where, const int64_t **ids, const double **dist2, int32_t *k, int64_t *nq)
{
    if (!r || r->kind != 1) {
        set_error("dl_result_topk: not a top-k result");
        return DL_EINVAL;
    }
    if (k) *k = r->k;
    if (nq) *nq = r->nq;
    if (where == DL_MEM_DEVICE) {
        if (ids) *ids = r->d_ids;
        if (dist2) *dist2 = r->d_d2;
        return DL_OK;
    }
    if (where != DL_MEM_HOST) {
        set_error("dl_result_topk: bad memory kind");
        return DL_EINVAL;
    }
    if (!r->h_ids) {
        const size_t n = (size_t)r->nq * r->k;
        size_t got = 0;
        void *h = hpool_get(std::max<size_t>(16, n * 16), &got);
        if (!h) {
            set_error("dl_result_topk: pinned host allocation failed");
            return DL_ENOMEM;
        }
        r->h_ids = (int64_t *)h;
        r->h_d2 = (double *)(r->h_ids + n);
        r->h_bytes = got;
        cudaError_t e = cudaSuccess;
        if (n > 0) e = cudaMemcpyAsync(r->h_ids, r->d_ids, n * 8, cudaMemcpyDeviceToHost, r->stream);
        if (e == cudaSuccess && n > 0) e = cudaMemcpyAsync(r->h_d2, r->d_d2, n * 8, cudaMemcpyDeviceToHost, r->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
        if (e != cudaSuccess) return cuda_fail(e, "dl_result_topk copy");
    }
    if (ids) *ids = r->h_ids;
    if (dist2) *dist2 = r->h_d2;
    return DL_OK;
}

int dl_result_stats(const dl_result *r, dl_join_stats *st)
{
    if (!r || !st) {
        set_error("dl_result_stats: NULL argument");
        return DL_EINVAL;
    }
    *st = r->stats;
    return DL_OK;
}

int dl_result_free(dl_result *r)
{
    if (!r) return DL_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != r->device) cudaSetDevice(r->device);
    if (r->kind == 0 || r->kind == 2) dev_free(r->d_r, r->stream);    // d_s lives in the same block
    if (r->kind == 1 || r->kind == 2) dev_free(r->d_ids, r->stream);  // d_d2 lives in the same block
    if (prev != r->device) cudaSetDevice(prev);
    if (r->h_r) hpool_put(r->h_r, r->h_bytes);
    if (r->kind == 1 && r->h_ids) hpool_put(r->h_ids, r->h_bytes);
    if (r->kind == 2 && r->h_batch) hpool_put(r->h_batch, r->h_batch_bytes);
    delete r;
    return DL_OK;
}

// Host copy of a batch result's pair arrays (all requests) on first use.
static int batch_pairs_host(dl_result *r)
{
    if (r->h_r) return DL_OK;
    const int64_t cnt = r->count;
    size_t got = 0;
    void *h = hpool_get(std::max<size_t>(16, (size_t)cnt * 16), &got);
    if (!h) {
        set_error("batch result: pinned host allocation failed");
        return DL_ENOMEM;
    }
    r->h_r = (int64_t *)h;
    r->h_s = r->h_r + cnt;
    r->h_bytes = got;
    cudaError_t e = cudaSuccess;
    if (cnt > 0) e = cudaMemcpyAsync(r->h_r, r->d_r, cnt * 8, cudaMemcpyDeviceToHost, r->stream);
    if (e == cudaSuccess && cnt > 0) e = cudaMemcpyAsync(r->h_s, r->d_s, cnt * 8, cudaMemcpyDeviceToHost, r->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch result copy");
    return DL_OK;
}

static int batch_topk_host(dl_result *r)
{
    if (r->h_batch) return DL_OK;
    const int64_t n = r->n_topk_slots;
    size_t got = 0;
    void *h = hpool_get(std::max<size_t>(16, (size_t)n * 16), &got);
    if (!h) {
        set_error("batch result: pinned host allocation failed");
        return DL_ENOMEM;
    }
    r->h_batch = h;
    r->h_batch_bytes = got;
    cudaError_t e = cudaSuccess;
    if (n > 0) e = cudaMemcpyAsync(h, r->d_ids, n * 8, cudaMemcpyDeviceToHost, r->stream);
    if (e == cudaSuccess && n > 0)
        e = cudaMemcpyAsync((char *)h + n * 8, r->d_d2, n * 8, cudaMemcpyDeviceToHost, r->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch result copy");
    return DL_OK;
}

int dl_result_request_pairs(dl_result *r, int32_t req, int32_t where, const int64_t **r_ids, const int64_t **s_ids,
                            int64_t *n)
{
    if (!r || r->kind != 2 || req < 0 || req >= (int32_t)r->req_kind.size() || r->req_kind[req] != DL_REQ_EPS) {
        set_error("dl_result_request_pairs: not an epsilon-join request of a batch result");
        return DL_EINVAL;
    }
    const int64_t o = r->pair_off[req], c = r->pair_off[req + 1] - o;
    if (n) *n = c;
    if (where == DL_MEM_DEVICE) {
        if (r_ids) *r_ids = r->d_r ? r->d_r + o : nullptr;
        if (s_ids) *s_ids = r->d_s ? r->d_s + o : nullptr;
        return DL_OK;
    }
    if (where != DL_MEM_HOST) {
        set_error("dl_result_request_pairs: bad memory kind");
        return DL_EINVAL;
    }
    const int rc = batch_pairs_host(r);
    if (rc) return rc;
    if (r_ids) *r_ids = r->h_r + o;
    if (s_ids) *s_ids = r->h_s + o;
    return DL_OK;
}

int dl_result_request_topk(dl_result *r, int32_t req, int32_t where, const int64_t **ids, const double **dist2,
                           int32_t *k, int64_t *nq)
{
    if (!r || r->kind != 2 || req < 0 || req >= (int32_t)r->req_kind.size() || r->req_kind[req] != DL_REQ_TOPK) {
        set_error("dl_result_request_topk: not a top-k request of a batch result");
        return DL_EINVAL;
    }
    const int64_t o = r->topk_off[req];
    if (k) *k = r->req_k[req];
    if (nq) *nq = r->req_nq[req];
    if (where == DL_MEM_DEVICE) {
        if (ids) *ids = r->d_ids ? r->d_ids + o : nullptr;
        if (dist2) *dist2 = r->d_d2 ? r->d_d2 + o : nullptr;
        return DL_OK;
    }
    if (where != DL_MEM_HOST) {
        set_error("dl_result_request_topk: bad memory kind");
        return DL_EINVAL;
    }
    const int rc = batch_topk_host(r);
    if (rc) return rc;
    const int64_t *hi = (const int64_t *)r->h_batch;
    const double *hd = (const double *)((const char *)r->h_batch + r->n_topk_slots * 8);
    if (ids) *ids = hi + o;
    if (dist2) *dist2 = hd + o;
    return DL_OK;
}

int dl_debug_check_word(uint64_t *word)
{
    clear_error();
    if (!word) {
        set_error("dl_debug_check_word: word is NULL");
        return DL_EINVAL;
    }
    *word = 0;
    int (*readers[])(unsigned long long *) = {check_read_api, check_read_join_tc, check_read_topk, check_read_recheck,
                                              check_read_batch};
    for (auto rd : readers) {
        unsigned long long w = 0;
        const int e = rd(&w);
        if (e) return cuda_fail((cudaError_t)e, "dl_debug_check_word");
        if (!*word) *word = w;
    }
    return DL_OK;
}

int dl_debug_check_selftest(int64_t index)
{
    clear_error();
#ifdef DL_CHECKED
    k_check_selftest<<<1, 1>>>((long long)index);
    DL_CUDA_TRY(cudaGetLastError());
    DL_CUDA_TRY(cudaDeviceSynchronize());
    return DL_OK;
#else
    (void)index;
    set_error("dl_debug_check_selftest: this library was built without DL_CHECKED");
    return DL_EUNSUPPORTED;
#endif
}

}  // extern "C"
