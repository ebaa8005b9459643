// hist_topk.cu -- the top-k join under the histogram distances (L1, chi-square): for every query
// row, the k store rows with the smallest canonical distance, ordered by (distance, store row)
// (Sec. 6.2 q1 -- the closest images to a query image -- with the colour-histogram distances of
// Sec. 4.1). These distances are not contractions, so they run on the CUDA cores.
//
// One CTA per query row (rows in chunks that bound the scratch memory):
//   1. the FP32 distance to every store row, one warp per store row, with its bound
//      |D32 - D| <= g32 D + a32 (the L1 / chi-square SIMT join's bound, which holds for any
//      summation order of the non-negative terms) -> lower and upper bounds;
//   2. the k-th smallest upper bound by a radix select over the float bits;
//   3. every store row whose lower bound reaches it (widened by the canonical sum's slack);
//   4. their canonical FP64 distances (k ascending, every operation rounded to nearest:
//      t = q_k - x_k, then s += |t| (L1), or u = q_k + x_k and, where u > 0, s += t*t / u);
//   5. the exact rank by (canonical distance, caller's store row); rank < k is written.
#include <algorithm>

#include "kernels.h"

namespace dl {

namespace {

constexpr int kHtCap = 8192;   // candidates a row can rank (more: DL_EOVERFLOW, many exact ties)

struct HistTk {
    const float *Q, *S;
    int d, nS, k;
    int64_t row0, nQ;
    float *scr_u, *scr_l;     // [rows][nS]
    uint32_t *scr_c;          // [rows][kHtCap]
    double *scr_d;            // [rows][kHtCap]
    const int32_t *q_orig, *s_orig;
    const int64_t *s_ids;
    int64_t *out_ids;
    double *out_d;
    float g32, a32, slack;
    int *err;
    unsigned long long *n_fp64;
};

template <int M>
__device__ __forceinline__ float term32(float a, float b)
{
    const float t = a - b;
    if constexpr (M == 1) {
        return fabsf(t);
    } else {
        const float u = a + b;
        return u > 0.f ? __fdiv_rn(t * t, u) : 0.f;
    }
}

template <int M>
__device__ double canon_hist(const float *__restrict__ q, const float *__restrict__ x, int d)
{
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        const double a = (double)__ldg(q + k), b = (double)__ldg(x + k);
        const double t = __dsub_rn(a, b);
        if constexpr (M == 1) {
            s = __dadd_rn(s, fabs(t));
        } else {
            const double u = __dadd_rn(a, b);
            if (u > 0.0) s = __dadd_rn(s, __ddiv_rn(__dmul_rn(t, t), u));
        }
    }
    return s;
}

template <int M>
__global__ void __launch_bounds__(256) k_hist_topk(const HistTk f)
{
    __shared__ unsigned hist[256];
    __shared__ unsigned s_prefix, s_rank;
    __shared__ int s_m;
    const int b = blockIdx.x;
    const int64_t i = f.row0 + b;
    if (i >= f.nQ) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    float *u = f.scr_u + (size_t)b * f.nS;
    float *l = f.scr_l + (size_t)b * f.nS;
    uint32_t *cl = f.scr_c + (size_t)b * kHtCap;
    double *cd = f.scr_d + (size_t)b * kHtCap;
    const float *q = f.Q + (size_t)i * f.d;
    // 1. FP32 distance bounds to every store row
    for (int j = warp; j < f.nS; j += nw) {
        const float *x = f.S + (size_t)j * f.d;
        float s = 0.f;
        for (int k = lane; k < f.d; k += 32) s += term32<M>(__ldg(q + k), __ldg(x + k));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            u[j] = __fadd_ru(__fmul_ru(s, 1.0f + f.g32), f.a32);
            l[j] = __fsub_rd(__fmul_rd(s, 1.0f - f.g32), f.a32);
        }
    }
    __syncthreads();
    // 2. k-th smallest upper bound by radix select on the (non-negative) float bits
    float kth = __int_as_float(0x7f800000);
    if (f.nS > f.k) {
        if (tid == 0) {
            s_prefix = 0u;
            s_rank = (unsigned)(f.k - 1);
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
    // 3. every store row whose lower bound is within it
    if (tid == 0) s_m = 0;
    __syncthreads();
    for (int j = tid; j < f.nS; j += blockDim.x) {
        if (l[j] <= kth) {
            const int pos = atomicAdd(&s_m, 1);
            if (pos < kHtCap) cl[pos] = (uint32_t)j;
        }
    }
    __syncthreads();
    const int m = s_m;
    if (m > kHtCap) {
        if (tid == 0) atomicExch(f.err, 1);
        return;
    }
    // 4. canonical distances, 5. exact rank by (canonical distance, caller's store row)
    for (int a = tid; a < m; a += blockDim.x) cd[a] = canon_hist<M>(q, f.S + (size_t)cl[a] * f.d, f.d);
    if (tid == 0 && m) atomicAdd(f.n_fp64, (unsigned long long)m);
    __syncthreads();
    const int64_t base = (int64_t)f.q_orig[i] * f.k;
    for (int a = tid; a < m; a += blockDim.x) {
        const double da = cd[a];
        const int32_t oa = f.s_orig[cl[a]];
        int rank = 0;
        for (int bb = 0; bb < m; ++bb) {
            const double db = cd[bb];
            rank += (db < da) || (db == da && f.s_orig[cl[bb]] < oa);
        }
        if (rank < f.k) {
            f.out_ids[base + rank] = f.s_ids[cl[a]];
            f.out_d[base + rank] = da;
        }
    }
    for (int t = m + tid; t < f.k; t += blockDim.x) {
        f.out_ids[base + t] = -1;
        f.out_d[base + t] = -1.0;
    }
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

int hist_topk(const dl_store *Q, const dl_store *S, int metric, int k, int64_t *out_ids, double *out_d,
              cudaStream_t st, dl_join_stats *stats)
{
    const int d = Q->d;
    const int64_t nQ = Q->n, nS = S->n;
    if (nQ == 0) return DL_OK;
    // the SIMT join's bounds (|D32 - D| <= g32 D + a32) and the canonical sum's relative error g64
    const double g32 = metric == 1 ? (d + 4) * 1.1920928955078125e-07 : (d + 16) * 1.1920928955078125e-07;
    const double a32 = metric == 1 ? d * 7.52316384526264e-37 : d * 2.168404344971009e-19;   // d 2^-120, d 2^-62
    const double g64 = (metric == 1 ? d + 4 : d + 8) * 1.1102230246251565e-16;
    HistTk f{};
    f.Q = Q->x32;
    f.S = S->x32;
    f.d = d;
    f.nS = (int)nS;
    f.k = k;
    f.nQ = nQ;
    f.q_orig = Q->orig;
    f.s_orig = S->orig;
    f.s_ids = S->ids;
    f.out_ids = out_ids;
    f.out_d = out_d;
    f.g32 = f32_ru(g32);
    f.a32 = f32_ru(a32);
    f.slack = f32_ru(4.0 * g64 + 1e-12);   // (1 + g64) / (1 - g64) and this product's roundings
    // rows per launch: about 256 MB of scratch
    const size_t per_row = al256((size_t)std::max<int64_t>(nS, 1) * 8) + (size_t)kHtCap * 12;
    const int64_t rows = std::max<int64_t>(1, std::min<int64_t>(nQ, (int64_t)((size_t)(256u << 20) / per_row)));
    void *blk = nullptr;
    const size_t b_ul = al256((size_t)rows * std::max<int64_t>(nS, 1) * 8);
    const size_t b_c = al256((size_t)rows * kHtCap * 4), b_d = al256((size_t)rows * kHtCap * 8);
    int rc = dev_alloc(&blk, b_ul + b_c + b_d + 256, st);
    if (rc) return rc;
    f.scr_u = (float *)blk;
    f.scr_l = f.scr_u + (size_t)rows * std::max<int64_t>(nS, 1);
    f.scr_c = (uint32_t *)((char *)blk + b_ul);
    f.scr_d = (double *)((char *)blk + b_ul + b_c);
    int *err = (int *)((char *)blk + b_ul + b_c + b_d);
    unsigned long long *nf = (unsigned long long *)(err + 2);
    f.err = err;
    f.n_fp64 = nf;
    cudaError_t e = cudaMemsetAsync(err, 0, 16, st);
    for (int64_t r0 = 0; r0 < nQ && e == cudaSuccess; r0 += rows) {
        f.row0 = r0;
        const unsigned nb = (unsigned)std::min<int64_t>(rows, nQ - r0);
        if (metric == 1)
            k_hist_topk<1><<<nb, 256, 0, st>>>(f);
        else
            k_hist_topk<2><<<nb, 256, 0, st>>>(f);
        count_launch();
        e = cudaGetLastError();
    }
    int herr = 0;
    unsigned long long hf = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof herr, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hf, nf, sizeof hf, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(blk, st);
    if (e != cudaSuccess) return cuda_fail(e, "histogram top-k");
    if (herr) {
        set_error("dl_topk_join: more than %d columns tie within the bound of a row's k-th distance", kHtCap);
        return DL_EOVERFLOW;
    }
    if (stats) {
        stats->pairs_evaluated = nQ * nS;
        stats->fp64_pairs = (int64_t)hf;
        stats->precision = DL_PREC_FP32;
        stats->kernels_launched = (int32_t)((nQ + rows - 1) / rows);
    }
    return DL_OK;
}

}  // namespace dl
