// topk.cu -- the top-k join (K4 + K7): for every query row, the k store rows
// with the smallest canonical distance, ordered by (distance, store row).
//
// The paper's reverse-image-search query (Sec. 6.2, q1: the closest image to a
// query image) is the k = 1 case. Pipeline on the caller's stream:
//   k_rowpar_topk      per query row: the bound terms and the canonical slack;
//   tc_join_kernel<.., true>   the tensor-core pass with the top-k epilogue: per
//                      (row, S split, epilogue half) slot a running threshold
//                      theta (k-th largest lower bound of h = q.x - ||x||^2/2)
//                      and the list of every column whose upper bound reached it;
//   k_topk_finalize    per row, one warp: union of the slots' lists above the
//                      largest theta, FP32 distances with their error bound, the
//                      k-th smallest upper bound, then the canonical FP64
//                      distance of every column that can still be in the top k
//                      and an exact rank by (D64, caller's store row index);
//   k_topk_fallback    rows whose lists overflowed (many near-ties) or whose
//                      candidates exceed the finalize buffer: an exact scan of
//                      the whole store for that row (FP32 bound + radix select +
//                      FP64 + rank).
// Store rows are in norm order; outputs are written at the caller's row order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "checked.cuh"
#include "kernels.h"

namespace dl {

constexpr int kTkMax = 480;          // candidates a finalize warp holds in shared memory (5 CTAs per SM)
// Canonical FP64 sums are costed per warp instruction (the FP64 rate is low and a warp-wide
// instruction occupies the pipe whatever its active lanes), so the finalize batches them: a row
// with at most kTkPendRow columns left queues them, and one lane-parallel pass computes the
// queued columns of many rows (up to kTkPend columns of kTkPendRows rows) at once.
constexpr int kTkPend = 64;
constexpr int kTkPendRow = 32;
constexpr int kTkPendRows = 32;
constexpr int kTkFallbackCap = 8192; // candidates a fallback block can rank

struct TopkFin {
    const float *Q, *S;
    int d, nQ, nS, k, slots, cap;
    const float *theta;
    const float *heap;     // [rows][slots][k] each slot's k largest lower bounds
    const unsigned *row_theta;
    const int *cnt;
    const uint2 *list;
    int *overflow;
    const int32_t *q_orig, *s_orig;
    const int64_t *s_ids;
    int64_t *out_ids;
    double *out_d2;
    const int *row_k;      // per query row k (NULL: k for every row)
    const int64_t *row_off;// per query row first output slot (NULL: caller row * k)
    float g32, abs32;      // FP32 distance bound: |D32 - D| <= g32 * D + abs32
    float slack;           // canonical slack factor for the keep test (relative)
    unsigned long long *n_fp64;
};

__device__ __forceinline__ double canon_d64(const float *__restrict__ q, const float *__restrict__ x, int d)
{
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        const double t = __dsub_rn((double)__ldg(q + k), (double)__ldg(x + k));
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

__device__ __forceinline__ float seq_d32(const float *__restrict__ q, const float *__restrict__ x, int d)
{
    float s = 0.f;
    for (int k = 0; k < d; ++k) {
        const float t = __ldg(q + k) - __ldg(x + k);
        s = fmaf(t, t, s);
    }
    return s;
}

// k-th largest of n floats (by order code), found by one warp with a 4-pass
// radix select over 8-bit digits; -inf when n < k. hist: 256 words of shared memory.
__device__ float warp_kth_largest(const float *__restrict__ vals, int n, int k, unsigned *hist)
{
    const unsigned lane = threadIdx.x & 31;
    if (n < k) return __int_as_float(0xff800000);
    unsigned prefix = 0u, mask = 0u;
    unsigned rank = (unsigned)(k - 1);   // 0-based, counted from the largest
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int t = lane; t < 256; t += 32) hist[t] = 0u;
        __syncwarp();
        for (int i = lane; i < n; i += 32) {
            const unsigned c = float_order_code(vals[i]);
            if ((c & mask) == prefix) atomicAdd(&hist[(c >> shift) & 255u], 1u);
        }
        __syncwarp();
        unsigned digit = 0u, r2 = 0u;
        if (lane == 0) {
            unsigned acc = 0u;
            for (int dg = 255; dg >= 0; --dg) {
                if (acc + hist[dg] > rank) {
                    digit = (unsigned)dg;
                    r2 = rank - acc;
                    break;
                }
                acc += hist[dg];
            }
        }
        digit = __shfl_sync(0xffffffffu, digit, 0);
        rank = __shfl_sync(0xffffffffu, r2, 0);
        prefix |= digit << shift;
        mask |= 255u << shift;
        __syncwarp();
    }
    return float_from_order_code(prefix);
}

__global__ void __launch_bounds__(128) k_topk_finalize(const TopkFin f)
{
    __shared__ unsigned s_hist[4][256];
    __shared__ uint32_t s_col[4][kTkMax];
    __shared__ float s_u[4][kTkMax];
    __shared__ float s_l[4][kTkMax];
    __shared__ double s_d[4][kTkMax];
    __shared__ float s_kth[4];
    __shared__ int s_prow[4][kTkPend];       // queued columns: query row,
    __shared__ uint32_t s_pcol[4][kTkPend];  // store row
    __shared__ int2 s_pseg[4][kTkPendRows];  // queued rows: {query row, first entry | count << 16}
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    uint32_t *col = s_col[w];
    float *su = s_u[w], *sl = s_l[w];
    double *sd = s_d[w];
    int np = 0, ns = 0;   // queued columns and rows of this warp (warp-uniform)
    // The queued columns' canonical distances (one per lane), then each queued row's exact rank
    // by (D64, caller's store row) and its outputs. Uses sd as scratch.
    auto flush = [&]() {
        for (int e = lane; e < np; e += 32)
            sd[e] = canon_d64(f.Q + (size_t)s_prow[w][e] * f.d, f.S + (size_t)s_pcol[w][e] * f.d, f.d);
        __syncwarp();
        for (int g = 0; g < ns; ++g) {
            const int2 sg = s_pseg[w][g];
            const int i = sg.x, e0 = sg.y & 0xffff, n = sg.y >> 16;
            const int kk = f.row_k ? f.row_k[i] : f.k;
            const int64_t base = f.row_off ? f.row_off[i] : (int64_t)f.q_orig[i] * f.k;
            for (int a = lane; a < n; a += 32) {
                const double da = sd[e0 + a];
                const uint32_t ca = s_pcol[w][e0 + a];
                const int32_t oa = f.s_orig[ca];
                int rank = 0;
                for (int b = 0; b < n; ++b) {
                    const double db = sd[e0 + b];
                    rank += (db < da) || (db == da && f.s_orig[s_pcol[w][e0 + b]] < oa);
                }
                if (rank < kk) {
                    f.out_ids[base + rank] = f.s_ids[ca];
                    f.out_d2[base + rank] = da;
                }
            }
            for (int t = n + lane; t < kk; t += 32) {
                f.out_ids[base + t] = -1;
                f.out_d2[base + t] = -1.0;
            }
        }
        __syncwarp();
        np = 0;
        ns = 0;
    };
    for (int i = blockIdx.x * 4 + w; i < f.nQ; i += gridDim.x * 4) {
        if (f.overflow[i]) continue;
        // the row's k-th largest lower bound over all slots' heaps (the heaps hold each
        // slot's k largest): every top-k column has U >= it
        const int kk0 = f.row_k ? f.row_k[i] : f.k;
        float th = warp_kth_largest(f.heap + (size_t)i * f.slots * f.k, f.slots * f.k, kk0, s_hist[w]);
        for (int s = lane; s < f.slots; s += 32) th = fmaxf(th, f.theta[(size_t)i * f.slots + s]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) th = fmaxf(th, __shfl_xor_sync(0xffffffffu, th, o));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) th = fmaxf(th, __shfl_xor_sync(0xffffffffu, th, o));
        int m = 0;
        for (int s = 0; s < f.slots; ++s) {
            const size_t si = (size_t)i * f.slots + s;
            const int cs = f.cnt[si];
            const uint2 *L = f.list + si * (size_t)f.cap;
            for (int b = 0; b < cs; b += 32) {
                const int idx = b + lane;
                uint2 e = make_uint2(0u, 0u);
                if (idx < cs) e = L[idx];
                const bool keep = idx < cs && __uint_as_float(e.y) >= th;
                const unsigned bm = __ballot_sync(0xffffffffu, keep);
                const int pos = m + __popc(bm & lt);
                if (keep && pos < kTkMax) col[pos] = DL_CHECK(e.x < (unsigned)f.nS, 10, e.x) ? e.x : 0u;
                m += __popc(bm);
            }
        }
        if (m > kTkMax) {   // too many candidates for this buffer: exact fallback
            if (lane == 0) f.overflow[i] = 1;
            continue;
        }
        __syncwarp();
        const float *q = f.Q + (size_t)i * f.d;
        for (int a = lane; a < m; a += 32) {
            const float d32 = seq_d32(q, f.S + (size_t)col[a] * f.d, f.d);
            su[a] = __fadd_ru(__fmul_ru(d32, 1.0f + f.g32), f.abs32);
            sl[a] = __fsub_rd(__fmul_rd(d32, 1.0f - f.g32), f.abs32);
        }
        __syncwarp();
        // k-th smallest upper bound (ties broken by position) -> at least k columns have D <= kth
        if (lane == 0) s_kth[w] = __int_as_float(0x7f800000);
        __syncwarp();
        const int kk = f.row_k ? f.row_k[i] : f.k;
        if (m > kk) {
            for (int a = lane; a < m; a += 32) {
                int rank = 0;
                const float ua = su[a];
                for (int b = 0; b < m; ++b) rank += (su[b] < ua) || (su[b] == ua && b < a);
                if (rank == kk - 1) s_kth[w] = ua;
            }
        }
        __syncwarp();
        const float kth = __fmul_ru(s_kth[w], 1.0f + f.slack);
        // the columns that can still be in the top k: each needs its canonical distance
        int kept = 0;
        for (int a0 = 0; a0 < m; a0 += 32) kept += __popc(__ballot_sync(0xffffffffu, a0 + lane < m && sl[a0 + lane] <= kth));
        if (lane == 0 && kept) atomicAdd(f.n_fp64, (unsigned long long)kept);
        if (kept <= kTkPendRow) {   // queue them with other rows' columns
            if (np + kept > kTkPend || ns == kTkPendRows) flush();
            int pos = np;
            for (int a0 = 0; a0 < m; a0 += 32) {
                const int a = a0 + lane;
                const bool keep = a < m && sl[a] <= kth;
                const unsigned bm = __ballot_sync(0xffffffffu, keep);
                if (keep) {
                    s_prow[w][pos + __popc(bm & lt)] = i;
                    s_pcol[w][pos + __popc(bm & lt)] = col[a];
                }
                pos += __popc(bm);
            }
            if (lane == 0) s_pseg[w][ns] = make_int2(i, np | (kept << 16));
            np += kept;
            ++ns;
            __syncwarp();
            continue;
        }
        flush();   // sd is this row's now
        for (int a0 = 0; a0 < m; a0 += 32) {
            const int a = a0 + lane;
            const bool keep = a < m && sl[a] <= kth;
            if (a < m) sd[a] = keep ? canon_d64(q, f.S + (size_t)col[a] * f.d, f.d) : __longlong_as_double(0x7ff0000000000000LL);
        }
        __syncwarp();
        const int64_t base = f.row_off ? f.row_off[i] : (int64_t)f.q_orig[i] * f.k;
        int64_t *oid = f.out_ids + base;
        double *od = f.out_d2 + base;
        for (int a = lane; a < m; a += 32) {
            const double da = sd[a];
            if (!(da < __longlong_as_double(0x7ff0000000000000LL))) continue;   // not kept
            const int32_t oa = f.s_orig[col[a]];
            int rank = 0;
            for (int b = 0; b < m; ++b) {
                const double db = sd[b];
                rank += (db < da) || (db == da && f.s_orig[col[b]] < oa);
            }
            if (rank < kk) {
                oid[rank] = f.s_ids[col[a]];
                od[rank] = da;
            }
        }
        for (int t = kept + lane; t < kk; t += 32) {
            oid[t] = -1;
            od[t] = -1.0;
        }
        __syncwarp();
    }
    flush();
}

struct TopkFb {
    const float *Q, *S;
    int d, nS, k;
    const int *rows;        // flagged query rows (store order)
    int n_rows;
    float *scr_u, *scr_l;   // [n_rows][nS]
    uint32_t *scr_c;        // [n_rows][kTkFallbackCap]
    double *scr_d;          // [n_rows][kTkFallbackCap]
    const int32_t *q_orig, *s_orig;
    const int64_t *s_ids;
    int64_t *out_ids;
    double *out_d2;
    const int *row_k;
    const int64_t *row_off;
    float g32, abs32, slack;
    int *err;               // set to 1 when a row has more near-ties than the fallback can rank
    unsigned long long *n_fp64;
};

// One block per flagged row: exact scan of the whole store.
__global__ void __launch_bounds__(256) k_topk_fallback(const TopkFb f)
{
    __shared__ unsigned hist[256];
    __shared__ unsigned s_prefix, s_rank;
    __shared__ int s_m;
    const int b = blockIdx.x;
    if (b >= f.n_rows) return;
    const int i = f.rows[b];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    float *u = f.scr_u + (size_t)b * f.nS;
    float *l = f.scr_l + (size_t)b * f.nS;
    uint32_t *cl = f.scr_c + (size_t)b * kTkFallbackCap;
    double *cd = f.scr_d + (size_t)b * kTkFallbackCap;
    const float *q = f.Q + (size_t)i * f.d;
    // 1. FP32 distance bounds to every store row
    for (int j = warp; j < f.nS; j += nw) {
        const float *x = f.S + (size_t)j * f.d;
        float s = 0.f;
        for (int k = lane; k < f.d; k += 32) {
            const float t = __ldg(q + k) - __ldg(x + k);
            s = fmaf(t, t, s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            u[j] = __fadd_ru(__fmul_ru(s, 1.0f + f.g32), f.abs32);
            l[j] = __fsub_rd(__fmul_rd(s, 1.0f - f.g32), f.abs32);
        }
    }
    __syncthreads();
    // 2. k-th smallest upper bound by radix select on the (non-negative) float bits
    const int kk = f.row_k ? f.row_k[i] : f.k;
    float kth = __int_as_float(0x7f800000);
    if (f.nS > kk) {
        if (tid == 0) {
            s_prefix = 0u;
            s_rank = (unsigned)(kk - 1);
        }
        for (int shift = 24; shift >= 0; shift -= 8) {
            for (int t = tid; t < 256; t += blockDim.x) hist[t] = 0u;
            __syncthreads();
            const unsigned pre = s_prefix;
            const unsigned mask_hi = (shift == 24) ? 0u : (0xffffffffu << (shift + 8));
            for (int j = tid; j < f.nS; j += blockDim.x) {
                const unsigned v = __float_as_uint(u[j]);
                if ((v & mask_hi) == (pre & mask_hi)) atomicAdd(&hist[(v >> shift) & 255u], 1u);
            }
            __syncthreads();
            if (tid == 0) {
                unsigned r = s_rank, acc = 0u;
                int dg = 0;
                for (; dg < 256; ++dg) {
                    if (acc + hist[dg] > r) break;
                    acc += hist[dg];
                }
                s_rank = r - acc;
                s_prefix = pre | ((unsigned)dg << shift);
            }
            __syncthreads();
        }
        kth = __uint_as_float(s_prefix);
    }
    kth = __fmul_ru(kth, 1.0f + f.slack);
    // 3. every row whose lower bound is within the k-th upper bound
    if (tid == 0) s_m = 0;
    __syncthreads();
    for (int j = tid; j < f.nS; j += blockDim.x) {
        if (l[j] <= kth) {
            const int pos = atomicAdd(&s_m, 1);
            if (pos < kTkFallbackCap) cl[pos] = (uint32_t)j;
        }
    }
    __syncthreads();
    const int m = s_m;
    if (m > kTkFallbackCap) {
        if (tid == 0) atomicExch(f.err, 1);
        return;
    }
    // 4. canonical distances, 5. exact rank by (D64, caller's store row)
    for (int a = tid; a < m; a += blockDim.x) cd[a] = canon_d64(q, f.S + (size_t)cl[a] * f.d, f.d);
    if (tid == 0) atomicAdd(f.n_fp64, (unsigned long long)m);
    __syncthreads();
    const int64_t base = f.row_off ? f.row_off[i] : (int64_t)f.q_orig[i] * f.k;
    int64_t *oid = f.out_ids + base;
    double *od = f.out_d2 + base;
    for (int a = tid; a < m; a += blockDim.x) {
        const double da = cd[a];
        const int32_t oa = f.s_orig[cl[a]];
        int rank = 0;
        for (int bb = 0; bb < m; ++bb) {
            const double db = cd[bb];
            rank += (db < da) || (db == da && f.s_orig[cl[bb]] < oa);
        }
        if (rank < kk) {
            oid[rank] = f.s_ids[cl[a]];
            od[rank] = da;
        }
    }
    for (int t = m + tid; t < kk; t += blockDim.x) {
        oid[t] = -1;
        od[t] = -1.0;
    }
}

// Per query row: {canonical slack of h, unused, ||q - q~|| up, ||q~|| up}; padding rows get zeros.
__global__ void __launch_bounds__(256) k_rowpar_topk(const double *__restrict__ nq64, const float4 *__restrict__ rowb,
                                                     int64_t n, int64_t n_tot, double g64, double nq_max_s,
                                                     float4 *__restrict__ rowpar, unsigned *__restrict__ row_theta)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_tot) return;
    row_theta[i] = float_order_code(__int_as_float(0xff800000));   // -inf
    if (i >= n) {
        rowpar[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    // |h_canonical - h| <= |D64 - D| / 2 <= g64 * (||q||^2 + ||x||^2); doubled for margin
    const double delta = 2.0 * g64 * (nq64[i] + nq_max_s) * 1.0001 + 1e-30;
    const float4 rb = rowb[i];
    rowpar[i] = make_float4(__double2float_ru(delta), 0.f, rb.x, rb.y);
}

__global__ void k_collect_overflow(const int *__restrict__ overflow, int n, int *__restrict__ rows,
                                   int *__restrict__ count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && overflow[i]) rows[atomicAdd(count, 1)] = i;
}

// ------------------------------------------------------------------ units with S splits
static std::mutex g_tku_mu;
static std::map<std::tuple<int, int64_t, int64_t, int, int>, std::pair<int4 *, int>> g_tku;

static int topk_units(int64_t nQ, int64_t nS, int BN, int splits, const int4 **d_units, int *n_units)
{
    int dev = 0;
    cudaGetDevice(&dev);
    auto key = std::make_tuple(dev, nQ, nS, BN, splits);
    std::lock_guard<std::mutex> lk(g_tku_mu);
    auto it = g_tku.find(key);
    if (it == g_tku.end()) {
        const int mt = (int)((nQ + 127) / 128), nt = (int)((nS + BN - 1) / BN);
        std::vector<int4> v;
        // split-major: the CTAs running together walk the same S range (shared through L2),
        // and later splits of a row start from the threshold its earlier splits published
        for (int s = 0; s < splits; ++s)
            for (int m = 0; m < mt; ++m) {
                const int nb = (int)((int64_t)nt * s / splits), ne = (int)((int64_t)nt * (s + 1) / splits);
                if (ne > nb) v.push_back(make_int4(m, nb, ne, s));
            }
        int4 *d = nullptr;
        if (!v.empty()) {
            cudaError_t e = cudaMalloc(&d, v.size() * sizeof(int4));
            if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(topk units)");
            e = cudaMemcpy(d, v.data(), v.size() * sizeof(int4), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(topk units)");
        }
        it = g_tku.emplace(key, std::make_pair(d, (int)v.size())).first;
    }
    *d_units = it->second.first;
    *n_units = it->second.second;
    return DL_OK;
}

static size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// Top-k of every row of Q against S into out_ids / out_d2. k is the largest k of
// any row (the heap size); row_k (device, optional) gives each row's own k and
// row_off (device, optional) each row's first output slot (default: caller row * k).
int topk_core(const dl_store *Q, const dl_store *S, int k, const int *row_k, const int64_t *row_off,
              int64_t *out_ids, double *out_d2, const dl_join_opts &o, cudaStream_t st, dl_join_stats *stats)
{
    const int64_t nQ = Q->n, nS = S->n;
    const int d = Q->d;
    if (o.tile_n != 0 && o.tile_n != 128 && o.tile_n != 256) {
        set_error("top-k: tile_n must be 0, 128 or 256");
        return DL_EINVAL;
    }
    const bool use_tc = (o.precision != DL_PREC_FP32) && Q->dp <= 512;
    bool tune_trial = false;
    if ((o.epilogue_warps != 0 && o.epilogue_warps != 8 && o.epilogue_warps != 16) ||
        (o.epilogue_warps == 16 && o.tile_n == 128)) {
        set_error("top-k: epilogue_warps must be 0, 8 or 16 (16: tile_n 0 or 256)");
        return DL_EINVAL;
    }
    int code = (o.tile_n ? o.tile_n : 256) | (o.epilogue_warps == 16 ? kTuneWide : 0);
    if (use_tc && o.tile_n == 0 && o.epilogue_warps == 0) code = tune_pick(Q->dp, kTuneTopk, nQ, nS, &tune_trial);
    const int BN = tune_bn(code);
    const bool wide = use_tc && tune_wide(code);   // 16 epilogue warps: slots per (row, split, quarter)
    const int sms = device_sm_count();
    const int64_t mt = (nQ + 127) / 128, nt = (nS + BN - 1) / BN;
    int splits = 1;
    if (mt > 0) splits = (int)std::min<int64_t>(std::max<int64_t>(1, (2 * sms + mt - 1) / mt), std::min<int64_t>(nt, 16));
    if (splits < 1) splits = 1;
    const int slots = (wide ? 4 : 2) * splits;
    const int cap = std::max(64, (4 * k + 31) / 32 * 32);
    const int64_t rows = mt * 128;

    const size_t b_rowpar = al256(rows * sizeof(float4)), b_heap = al256((size_t)rows * slots * k * sizeof(float)),
                 b_list = al256((size_t)rows * slots * cap * sizeof(uint2)),
                 b_cnt = al256((size_t)rows * slots * sizeof(int)), b_theta = al256((size_t)rows * slots * sizeof(float)),
                 b_rth = al256((size_t)std::max<int64_t>(rows, 1) * sizeof(unsigned)),
                 b_ovf = al256((size_t)std::max<int64_t>(nQ, 1) * sizeof(int)),
                 b_rows = al256((size_t)std::max<int64_t>(nQ, 1) * sizeof(int)), b_misc = 256;
    const bool timing = o.timing || tune_trial;
    void *ws = nullptr;
    int rc = dev_alloc(&ws, b_rowpar + b_heap + b_list + b_cnt + b_theta + b_rth + b_ovf + b_rows + b_misc, st);
    if (rc) return rc;
    char *pw = (char *)ws;
    float4 *rowpar = (float4 *)pw;
    pw += b_rowpar;
    float *heap = (float *)pw;
    pw += b_heap;
    uint2 *list = (uint2 *)pw;
    pw += b_list;
    int *cnt = (int *)pw;
    pw += b_cnt;
    float *theta = (float *)pw;
    pw += b_theta;
    unsigned *row_theta = (unsigned *)pw;
    pw += b_rth;
    int *ovf = (int *)pw;
    pw += b_ovf;
    int *frows = (int *)pw;
    pw += b_rows;
    unsigned long long *misc = (unsigned long long *)pw;   // [0] flagged rows [1] fp64 evals [2] err [3] tc err
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    if (timing)
        for (auto &e : ev) cudaEventCreate(&e);
    auto done = [&](int code) {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
        dev_free(ws, st);
        if (code) cudaStreamSynchronize(st);
        return code;
    };
    cudaError_t e = cudaMemsetAsync(misc, 0, 256, st);
    if (e == cudaSuccess && nQ > 0) e = cudaMemsetAsync(ovf, 0, (size_t)nQ * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, b_cnt, st);
    if (e != cudaSuccess) return done(cuda_fail(e, "top-k memset"));
    if (timing) cudaEventRecord(ev[0], st);
    int launches = 0;
    const double g64 = gamma64(d), g32 = gamma32(d);
    TopkFin f;
    f.Q = Q->x32;
    f.S = S->x32;
    f.d = d;
    f.nQ = (int)nQ;
    f.nS = (int)nS;
    f.k = k;
    f.slots = slots;
    f.cap = cap;
    f.theta = theta;
    f.heap = heap;
    f.row_theta = row_theta;
    f.cnt = cnt;
    f.list = list;
    f.overflow = ovf;
    f.q_orig = Q->orig;
    f.s_orig = S->orig;
    f.s_ids = S->ids;
    f.out_ids = out_ids;
    f.out_d2 = out_d2;
    f.row_k = row_k;
    f.row_off = row_off;
    f.g32 = f32_ru(g32 * 1.0000001);
    f.abs32 = f32_ru((double)(d + 8) * 1.401298464324817e-45 * 4.0);
    f.slack = f32_ru(4.0 * g64 + 1e-12);
    f.n_fp64 = misc + 1;
    if (nQ > 0 && nS > 0) {
        if (use_tc) {
            k_rowpar_topk<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(Q->nq64, Q->rowb, nQ, rows, g64,
                                                                          (double)S->nq_max * 1.0001, rowpar, row_theta);
            count_launch();
            ++launches;
            const CUtensorMap *tmA = nullptr, *tmB = nullptr;
            rc = get_tmap(const_cast<dl_store *>(Q), 128, &tmA);
            if (!rc) rc = get_tmap(const_cast<dl_store *>(S), BN, &tmB);
            const int4 *units = nullptr;
            int n_units = 0;
            if (!rc) rc = topk_units(nQ, nS, BN, splits, &units, &n_units);
            if (!rc && n_units > 0) {
                TcLaunch L;
                std::memset(&L.p, 0, sizeof L.p);
                L.tmA = tmA;
                L.tmB = tmB;
                L.BN = BN;
                L.grid = std::min(n_units, sms);
                L.p.units = units;
                L.p.n_units = n_units;
                L.p.nR = (int)nQ;
                L.p.nS = (int)nS;
                L.p.kc = Q->dp / 64;
                tc_plan(BN, Q->dp / 64, &L.p.stages, &L.p.a_slots, false, false, wide);
                L.wide = wide;
                L.p.upper = 0;
                L.p.rowpar = rowpar;
                L.p.beta = S->beta;
                L.p.cstat = S->cstat;
                L.p.err = (int *)(misc + 3);
                L.p.tk_k = k;
                L.p.tk_cap = cap;
                L.p.tk_slots = slots;
                L.p.tk_heap = heap;
                L.p.tk_list = list;
                L.p.tk_cnt = cnt;
                L.p.tk_theta = theta;
                L.p.tk_row_theta = row_theta;
                L.p.tk_overflow = ovf;
                // Units are split-major, so the first mt units are every row tile's first split.
                // Running those alone first publishes each row's threshold before the other
                // splits start: their slots then admit only columns that can still reach the
                // top k (fewer list entries and heap inserts, most visibly for large k).
                // (only when the first splits alone still fill most of the GPU)
                const int first = (splits > 1 && n_units > mt && 2 * mt >= sms) ? (int)mt : n_units;
                L.p.n_units = first;
                L.grid = std::min(first, sms);
                rc = launch_tc_join(L, st, true);
                ++launches;
                if (!rc && first < n_units) {
                    L.p.units = units + first;
                    L.p.n_units = n_units - first;
                    L.grid = std::min(n_units - first, sms);
                    rc = launch_tc_join(L, st, true);
                    ++launches;
                }
            }
            if (!rc) {
                const int grid = (int)std::min<int64_t>((nQ + 3) / 4, (int64_t)sms * 16);
                k_topk_finalize<<<grid, 128, 0, st>>>(f);
                count_launch();
                ++launches;
                e = cudaGetLastError();
                if (e != cudaSuccess) rc = cuda_fail(e, "k_topk_finalize launch");
            }
        } else {
            // no tensor-core pass for this shape: every row takes the exact scan
            e = cudaMemsetAsync(ovf, 0xff, (size_t)nQ * sizeof(int), st);
            if (e != cudaSuccess) rc = cuda_fail(e, "top-k memset");
        }
    } else if (nQ > 0) {   // empty store: every slot is unused
        k_rowpar_topk<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(Q->nq64, Q->rowb, nQ, rows, g64, 0.0, rowpar,
                                                                      row_theta);
        k_topk_finalize<<<1, 128, 0, st>>>(f);   // no candidates for any row -> fills -1
        count_launch();
        count_launch();
        ++launches;
    }
    if (timing) cudaEventRecord(ev[1], st);
    // exact fallback for flagged rows
    int64_t flagged = 0;
    if (!rc && nQ > 0 && nS > 0) {
        k_collect_overflow<<<(unsigned)((nQ + 255) / 256), 256, 0, st>>>(ovf, (int)nQ, frows, (int *)misc);
        count_launch();
        ++launches;
        unsigned long long h[4] = {0, 0, 0, 0};
        e = cudaMemcpyAsync(h, misc, sizeof h, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "top-k");
        if (!rc && h[3]) {
            set_error("top-k: a bounded device wait expired");
            return done(DL_ETIMEOUT);
        }
        flagged = (int64_t)(h[0] & 0xffffffffULL);
        if (!rc && flagged > 0) {
            const int64_t per_row = (int64_t)nS * 8 + (int64_t)kTkFallbackCap * 12;
            const int64_t batch = std::max<int64_t>(1, std::min<int64_t>(flagged, (256LL << 20) / per_row));
            void *fb = nullptr;
            rc = dev_alloc(&fb, al256(batch * (size_t)nS * 8) + al256(batch * (size_t)kTkFallbackCap * 12), st);
            if (!rc) {
                TopkFb g;
                g.Q = Q->x32;
                g.S = S->x32;
                g.d = d;
                g.nS = (int)nS;
                g.k = k;
                g.scr_u = (float *)fb;
                g.scr_l = g.scr_u + batch * nS;
                g.scr_c = (uint32_t *)((char *)fb + al256(batch * (size_t)nS * 8));
                g.scr_d = (double *)(g.scr_c + batch * kTkFallbackCap);
                g.q_orig = Q->orig;
                g.s_orig = S->orig;
                g.s_ids = S->ids;
                g.out_ids = out_ids;
                g.out_d2 = out_d2;
                g.row_k = row_k;
                g.row_off = row_off;
                g.g32 = f.g32;
                g.abs32 = f.abs32;
                g.slack = f.slack;
                g.err = (int *)(misc + 2);
                g.n_fp64 = misc + 1;
                for (int64_t b0 = 0; b0 < flagged && !rc; b0 += batch) {
                    g.rows = frows + b0;
                    g.n_rows = (int)std::min<int64_t>(batch, flagged - b0);
                    k_topk_fallback<<<g.n_rows, 256, 0, st>>>(g);
                    count_launch();
                    ++launches;
                    e = cudaGetLastError();
                    if (e != cudaSuccess) rc = cuda_fail(e, "k_topk_fallback launch");
                }
                dev_free(fb, st);
            }
        }
    }
    if (timing) cudaEventRecord(ev[2], st);
    unsigned long long h2[4] = {0, 0, 0, 0};
    if (!rc) {
        e = cudaMemcpyAsync(h2, misc, sizeof h2, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "top-k");
    }
    if (!rc && h2[2]) {
        set_error("top-k: more than %d store rows tie within rounding at the k-th distance of a query",
                  kTkFallbackCap);
        rc = DL_EUNSUPPORTED;
    }
    if (rc) return done(rc);
    if (stats) {
        dl_join_stats &s = *stats;
        s.pairs_evaluated = nQ * nS;
        s.pairs_out = 0;
        s.band_pairs = flagged;   // rows re-solved by the exact scan
        s.fp64_pairs = (int64_t)h2[1];
        s.precision = use_tc ? DL_PREC_BF16 : DL_PREC_FP32;
        s.tile_n = use_tc ? BN : 0;
        s.epilogue_warps = use_tc ? (wide ? 16 : 8) : 0;
        s.kernels_launched = launches;
        if (timing) {
            cudaEventElapsedTime(&s.ms_main, ev[0], ev[1]);
            cudaEventElapsedTime(&s.ms_recheck, ev[1], ev[2]);
            cudaEventElapsedTime(&s.ms_total, ev[0], ev[2]);
        }
    }
    if (tune_trial && flagged == 0) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        tune_record(Q->dp, kTuneTopk, nQ, nS, code, ms, (double)nQ * (double)nS);
    }
    return done(DL_OK);
}

}  // namespace dl

using namespace dl;

extern "C" int dl_topk_join(const dl_store *Q, const dl_store *S, int32_t metric, int32_t k, const dl_join_opts *opts,
                            dl_result **out)
{
    dl::NvtxScope nvtx_scope("dl_topk_join");
    clear_error();
    if (!out) {
        set_error("dl_topk_join: out is NULL");
        return DL_EINVAL;
    }
    *out = nullptr;
    if (!Q || !S) {
        set_error("dl_topk_join: NULL store");
        return DL_EINVAL;
    }
    const bool hist = metric == DL_METRIC_L1 || metric == DL_METRIC_CHI2;
    if (metric == DL_METRIC_COSINE) {   // the most similar rows are the nearest normalized rows
        if (!Q->unit || !S->unit) {
            set_error("dl_topk_join: the cosine metric needs stores made by dl_store_normalize");
            return DL_EINVAL;
        }
    } else if (metric != DL_METRIC_L2 && !hist) {
        set_error("dl_topk_join: unsupported metric %d", metric);
        return DL_EINVAL;
    }
    if (k < 1 || k > 1024) {
        set_error("dl_topk_join: k=%d out of range [1, 1024]", k);
        return DL_EINVAL;
    }
    if (Q->d != S->d) {
        set_error("dl_topk_join: dimension mismatch %d vs %d", Q->d, S->d);
        return DL_EINVAL;
    }
    int dev = -1;
    DL_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != Q->device || dev != S->device) {
        set_error("dl_topk_join: stores live on another device");
        return DL_EINVAL;
    }
    dl_join_opts o;
    if (opts)
        o = *opts;
    else
        dl_join_opts_default(&o);
    if (o.precision != DL_PREC_AUTO && o.precision != DL_PREC_BF16 && o.precision != DL_PREC_FP32) {
        set_error("dl_topk_join: precision %d not available for top-k", o.precision);
        return DL_EUNSUPPORTED;
    }
    cudaStream_t st = (cudaStream_t)o.cuda_stream;
    if (hist && o.precision == DL_PREC_BF16) {
        set_error("dl_topk_join: the L1 and chi-square distances run in DL_PREC_FP32 (not on tensor cores)");
        return DL_EUNSUPPORTED;
    }
    int rc = DL_OK;
    if (metric == DL_METRIC_CHI2) {
        bool ok = false;
        rc = store_nonneg(const_cast<dl_store *>(Q), st, &ok);
        if (!rc && ok) rc = store_nonneg(const_cast<dl_store *>(S), st, &ok);
        if (rc) return rc;
        if (!ok) {
            set_error("dl_topk_join: the chi-square distance needs non-negative features");
            return DL_EINVAL;
        }
    }
    const int64_t nQ = Q->n;
    void *resb = nullptr;
    rc = dev_alloc(&resb, std::max<size_t>(16, (size_t)nQ * k * 16), st);
    if (rc) return rc;
    int64_t *out_ids = (int64_t *)resb;
    double *out_d2 = (double *)(out_ids + (size_t)nQ * k);
    dl_join_stats stats{};
    if (hist)
        rc = hist_topk(Q, S, metric == DL_METRIC_L1 ? 1 : 2, k, out_ids, out_d2, st, &stats);
    else
        rc = topk_core(Q, S, k, nullptr, nullptr, out_ids, out_d2, o, st, &stats);
    if (rc) {
        dev_free(resb, st);
        return rc;
    }
    stats.pairs_out = nQ * std::min<int64_t>(k, S->n);
    dl_result *res = new dl_result();
    res->kind = 1;
    res->device = dev;
    res->stream = st;
    res->k = k;
    res->nq = nQ;
    res->d_ids = out_ids;
    res->d_d2 = out_d2;
    res->stats = stats;
    *out = res;
    return DL_OK;
}

DL_CHECK_READER(topk)
