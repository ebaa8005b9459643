// store.cu -- the device-resident patch store and its derivation pass (K1).
//
// A store keeps a patch collection resident on the GPU (the in-memory form of
// "materialize", Sec. 3.2 / Sec. 4.1 of the paper): int64 ids, the FP32
// feature rows (the ground truth), a zero-padded BF16 copy for the tensor
// cores, and per-row / per-32-row-chunk statistics from which the join
// kernels derive sound error bounds.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include <cuda_fp8.h>

#include "internal.h"

namespace dl {

// ------------------------------------------------------------------ errors
static thread_local std::string t_err;

void set_error(const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
}

void clear_error() { t_err.clear(); }

const char *last_error() { return t_err.c_str(); }

int cuda_fail(cudaError_t e, const char *what)
{
    set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
    return DL_ECUDA;
}

std::atomic<int64_t> g_launches{0};

// ------------------------------------------------------------------ pools
static std::mutex g_pool_mu;
static bool g_pool_ready[64];

int dev_alloc(void **p, size_t bytes, cudaStream_t st)
{
    int dev = 0;
    DL_CUDA_TRY(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64) {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (!g_pool_ready[dev]) {
            // Keep freed blocks in the pool so repeated calls do not return memory
            // to the driver (a per-process pool attribute).
            cudaMemPool_t pool;
            if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
                uint64_t thr = UINT64_MAX;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
            }
            g_pool_ready[dev] = true;
        }
    }
    if (bytes == 0) bytes = 256;
    cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        *p = nullptr;
        return DL_ENOMEM;
    }
    return DL_OK;
}

void dev_free(void *p, cudaStream_t st)
{
    if (p) cudaFreeAsync(p, st);
}

int device_sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// ------------------------------------------------------------------ K1
// One warp per row. Computes, from the FP32 row x:
//   nq64  = sum x_k^2 in FP64 (products exact, rounding only in the sum),
//   the BF16 copy x~ = RN_bf16(x) (zero padded to dp),
//   upper bounds of ||x - x~|| and ||x~|| (FP32 sums of squares rounded up at every
//   step, square roots rounded up), and of ||x|| (from the FP64 sum, inflated by the
//   sum and sqrt rounding),
//   beta = RN32(nq64 / 2) and an upper bound of |beta - ||x||^2 / 2|,
// and flags rows with a non-finite value or |x_k| > 2^40.
__global__ void __launch_bounds__(256) k1_norm_quant(const float *__restrict__ x32, int64_t n, int d, int dp,
                                                     __nv_bfloat16 *__restrict__ xb, double *__restrict__ nq64,
                                                     float *__restrict__ beta, float4 *__restrict__ rowb,
                                                     int *__restrict__ err)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = ((int64_t)blockIdx.x * 8 + warp) * 32;   // this warp's 32 rows
    if (row0 >= n) return;
    const int rows = (int)(n - row0 < 32 ? n - row0 : 32);
    // the sums of row r end in lane r, so the per-row tail (FP64, a square root) runs once per
    // 32 rows with every lane busy: a warp-wide FP64 instruction costs the same at one lane
    double m1 = 0.0;
    float m2 = 0.f, m3 = 0.f;
    bool mbad = false;
    for (int r = 0; r < rows; ++r) {
        const int64_t row = row0 + r;
        const float *xr = x32 + row * d;
        __nv_bfloat16 *br = xb + row * dp;
        double s1 = 0.0;
        float s2 = 0.f, s3 = 0.f;   // rounded up at every step: upper bounds of the exact sums
        bool bad = false;
        for (int k = lane; k < dp; k += 32) {
            const float v = (k < d) ? __ldg(xr + k) : 0.0f;
            if (!(fabsf(v) <= 1099511627776.0f)) bad = true;  // also catches NaN
            const __nv_bfloat16 b = __float2bfloat16_rn(v);
            br[k] = b;
            const float fb = __bfloat162float(b);
            const float e = v - fb;   // exact: x~ shares x's leading bits
            const double dv = (double)v;
            s1 = __dadd_rn(s1, __dmul_rn(dv, dv));
            s2 = __fmaf_ru(e, e, s2);
            s3 = __fmaf_ru(fb, fb, s3);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s1 = __dadd_rn(s1, __shfl_xor_sync(0xffffffffu, s1, o));
            s2 = __fadd_ru(s2, __shfl_xor_sync(0xffffffffu, s2, o));
            s3 = __fadd_ru(s3, __shfl_xor_sync(0xffffffffu, s3, o));
        }
        bad = __any_sync(0xffffffffu, bad);
        if (lane == r) {
            m1 = s1;
            m2 = s2;
            m3 = s3;
            mbad = bad;
        }
    }
    if (lane < rows) {
        const int64_t row = row0 + lane;
        const double s1 = m1;
        const float s2 = m2, s3 = m3;
        if (mbad) atomicOr(err, 1);
        // Any-order FP64 sum of dp non-negative exact terms: relative error <= (dp-1) 2^-53.
        const double fac = 1.0 + (double)(dp + 4) * 2.220446049250313e-16;
        const double grow = 1.0 + 8.881784197001252e-16;   // 1 + 2^-50 covers the sqrt / product roundings
        nq64[row] = s1;
        const float rq = __fsqrt_ru(s2);
        const float nqt = __fsqrt_ru(s3);
        const float nx = __double2float_ru(sqrt(s1 * fac) * grow);
        const double h = 0.5 * s1;
        const float bt = __double2float_rn(h);
        const float berr = __double2float_ru((fabs((double)bt - h) + h * (double)(dp + 2) * 2.220446049250313e-16) * grow);
        beta[row] = bt;
        rowb[row] = make_float4(rq, nqt, nx, berr);
    }
}

// One warp per 32-row chunk: column-side maxima of the BF16 error-bound terms,
//   P1 = max ||x||,   P2 = max ||x - x~|| + (gamma_tc + 1.01 u) max ||x~||,
//   P3 = max |beta err| + u max beta + absolute slack,
//   and the chunk's smallest beta (for the epilogue's whole-chunk reject test),
// so that for a query row q and any column x in the chunk the error of the
// epilogue value h = fl(A~ - beta) is at most  rq * P1 + ||q~|| * P2 + P3.
// Also fills beta's padding with +inf (padded columns can never match).
__global__ void __launch_bounds__(256) k1_chunk_stats(const float *__restrict__ beta_in, const float4 *__restrict__ rowb,
                                                      int64_t n, int64_t n_pad, float g2, float p3_abs,
                                                      float *__restrict__ beta, float4 *__restrict__ cstat)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t chunk = (int64_t)blockIdx.x * 8 + warp;
    if (chunk * 32 >= n_pad) return;
    const int64_t row = chunk * 32 + lane;
    float rq = 0.f, nqt = 0.f, nx = 0.f, berr = 0.f, bt = 0.f;
    float bmin = __int_as_float(0x7f800000);   // +inf: padding rows do not lower the chunk minimum
    if (row < n) {
        const float4 rb = rowb[row];
        rq = rb.x;
        nqt = rb.y;
        nx = rb.z;
        berr = rb.w;
        bt = fabsf(beta_in[row]);
        bmin = beta_in[row];
    } else {
        beta[row] = __int_as_float(0x7f800000);   // +inf
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rq = fmaxf(rq, __shfl_xor_sync(0xffffffffu, rq, o));
        nqt = fmaxf(nqt, __shfl_xor_sync(0xffffffffu, nqt, o));
        nx = fmaxf(nx, __shfl_xor_sync(0xffffffffu, nx, o));
        berr = fmaxf(berr, __shfl_xor_sync(0xffffffffu, berr, o));
        bt = fmaxf(bt, __shfl_xor_sync(0xffffffffu, bt, o));
        bmin = fminf(bmin, __shfl_xor_sync(0xffffffffu, bmin, o));
    }
    if (lane == 0) {
        const float p2 = __fmaf_ru(g2, nqt, rq);
        const float p3 = __fadd_ru(__fmaf_ru(5.9604644775390625e-08f, bt, berr), p3_abs);
        cstat[chunk] = make_float4(nx, p2, p3, bmin);
    }
}

// ------------------------------------------------------------------ norm ordering
// A store keeps its rows ordered by squared norm (a bucket sort into 65,536
// equal-width buckets between the smallest and largest norm; order inside a
// bucket is arbitrary). Neighbouring rows then have nearly equal ||x||^2/2, so
// the join epilogue can bound a whole 32-column chunk with the chunk's
// smallest beta. The caller's row index of every store row is kept (orig).
constexpr int kSortBuckets = 65536;
static size_t align256(size_t x);

__global__ void __launch_bounds__(256) k_sort_keys(const float *__restrict__ x, int64_t n, int d,
                                                   float *__restrict__ keys, unsigned *__restrict__ minmax)
{
    __shared__ unsigned s_min[8], s_max[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * 8 + warp;
    unsigned kmin = 0xffffffffu, kmax = 0u;
    if (row < n) {
        const float *xr = x + row * d;
        float s = 0.f;
        for (int k = lane; k < d; k += 32) {
            const float v = __ldg(xr + k);
            s = fmaf(v, v, s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (!(s <= 3.0e38f)) s = 3.0e38f;   // non-finite rows are rejected later; keep the key ordered
        if (lane == 0) keys[row] = s;
        kmin = kmax = __float_as_uint(s);   // non-negative floats order like their bits
    }
    if (lane == 0) {
        s_min[warp] = kmin;
        s_max[warp] = kmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {   // one atomic pair per block of eight rows
        for (int w = 1; w < 8; ++w) {
            kmin = min(kmin, s_min[w]);
            kmax = max(kmax, s_max[w]);
        }
        if (kmin != 0xffffffffu) {
            atomicMin(minmax + 0, kmin);
            atomicMax(minmax + 1, kmax);
        }
    }
}

__device__ __forceinline__ int sort_bucket(float k, const unsigned *minmax)
{
    const float lo = __uint_as_float(minmax[0]), hi = __uint_as_float(minmax[1]);
    if (!(hi > lo)) return 0;
    const float f = (k - lo) / (hi - lo) * (float)kSortBuckets;
    int b = (int)f;
    return b < 0 ? 0 : (b >= kSortBuckets ? kSortBuckets - 1 : b);
}

__global__ void __launch_bounds__(256) k_sort_hist(const float *__restrict__ keys, int64_t n,
                                                   const unsigned *__restrict__ minmax, unsigned *__restrict__ hist)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(hist + sort_bucket(keys[i], minmax), 1u);
}

// Exclusive prefix sum of the 65,536 bucket counts, one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_sort_scan(unsigned *__restrict__ hist)
{
    __shared__ unsigned part[1024];
    constexpr int kPer = kSortBuckets / 1024;
    const int t = threadIdx.x;
    unsigned loc = 0;
    for (int i = 0; i < kPer; ++i) loc += hist[t * kPer + i];
    part[t] = loc;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const unsigned v = (t >= off) ? part[t - off] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    unsigned run = part[t] - loc;
    for (int i = 0; i < kPer; ++i) {
        const unsigned c = hist[t * kPer + i];
        hist[t * kPer + i] = run;
        run += c;
    }
}

__global__ void __launch_bounds__(256) k_sort_scatter(const float *__restrict__ keys, int64_t n,
                                                      const unsigned *__restrict__ minmax, unsigned *__restrict__ offs,
                                                      int32_t *__restrict__ perm)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) perm[atomicAdd(offs + sort_bucket(keys[i], minmax), 1u)] = (int32_t)i;
}

// Store row i <- caller row perm[i] (features and id), one warp per row.
__global__ void __launch_bounds__(256) k_gather_rows(const float *__restrict__ src, const int64_t *__restrict__ src_ids,
                                                     const int32_t *__restrict__ perm, int64_t n, int d,
                                                     float *__restrict__ dst, int64_t *__restrict__ dst_ids,
                                                     int32_t *__restrict__ orig)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * 8 + warp;
    if (row >= n) return;
    const int32_t j = perm[row];
    const float *sr = src + (int64_t)j * d;
    float *dr = dst + row * d;
    for (int k = lane; k < d; k += 32) dr[k] = __ldg(sr + k);
    if (lane == 0) {
        dst_ids[row] = src_ids[j];
        orig[row] = j;
    }
}

// ------------------------------------------------------------------ FP8 copy
// Every 32-row chunk shares one power-of-two scale s: the largest over its rows of the
// power of two s_row with max|x| / s_row <= 448 (the largest finite e4m3). Codes are
// RN_e4m3(x / s) (x / s is exact, and max|x| / s <= 448 still holds in every row). One
// scale per chunk lets the epilogue bound a whole chunk from its raw accumulators:
// h_j = fl(A_j s_q s - beta_j) <= fl_ru(max_j A_j * s_q s - beta_min).

// One warp per row: the row's own scale s_row.
__global__ void __launch_bounds__(256) k1_fp8_row_scale(const float *__restrict__ x32, int64_t n, int d,
                                                        float *__restrict__ sc8)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * 8 + warp;
    if (row >= n) return;
    const float *xr = x32 + row * d;
    float mx = 0.f;
    for (int k = lane; k < d; k += 32) mx = fmaxf(mx, fabsf(__ldg(xr + k)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    float sc = 1.0f;
    if (mx > 0.f) {
        int e;
        const float m = frexpf(mx / 448.0f, &e);   // mx/448 = m 2^e, m in [0.5, 1)
        int c = (m == 0.5f) ? e - 1 : e;           // ceil(log2(mx / 448))
        if (c < -126) c = -126;
        sc = ldexpf(1.0f, c);
        while (mx / sc > 448.0f) sc *= 2.0f;
    }
    if (lane == 0) sc8[row] = sc;
}

// One warp per 32-row chunk: the chunk scale (the largest row scale), written to the chunk
// table and to every row of the chunk (1 on padding rows).
__global__ void __launch_bounds__(256) k1_fp8_chunk_scale(int64_t n, int64_t n_pad, float *__restrict__ sc8,
                                                          float *__restrict__ scc8)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t chunk = (int64_t)blockIdx.x * 8 + warp;
    if (chunk * 32 >= n_pad) return;
    const int64_t row = chunk * 32 + lane;
    float sc = row < n ? sc8[row] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sc = fmaxf(sc, __shfl_xor_sync(0xffffffffu, sc, o));
    if (sc == 0.f) sc = 1.0f;
    sc8[row] = row < n ? sc : 1.0f;
    if (lane == 0) scc8[chunk] = sc;
}

// One warp per row: codes with the row's (chunk) scale, and upper bounds of
// ||x - s*dec(codes)|| and ||s*dec(codes)|| (FP32 sums of squares rounded up at every step,
// square roots rounded up).
__global__ void __launch_bounds__(256) k1_fp8(const float *__restrict__ x32, int64_t n, int d, int dp8,
                                              const float *__restrict__ sc8, uint8_t *__restrict__ x8,
                                              float2 *__restrict__ rowb8)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * 8 + warp;
    if (row >= n) return;
    const float *xr = x32 + row * d;
    const float sc = sc8[row];
    uint8_t *br = x8 + row * dp8;
    float s2 = 0.f, s3 = 0.f;
    for (int k = lane; k < dp8; k += 32) {
        const float v = (k < d) ? __ldg(xr + k) : 0.0f;
        const __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(v / sc, __NV_SATFINITE, __NV_E4M3);
        br[k] = (uint8_t)q;
        const float dec = __half2float(__half(__nv_cvt_fp8_to_halfraw(q, __NV_E4M3))) * sc;   // exact
        const float e = v - dec;   // exact: |e| is below half an e4m3 step of v / s, times s
        s2 = __fmaf_ru(e, e, s2);
        s3 = __fmaf_ru(dec, dec, s3);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s2 = __fadd_ru(s2, __shfl_xor_sync(0xffffffffu, s2, o));
        s3 = __fadd_ru(s3, __shfl_xor_sync(0xffffffffu, s3, o));
    }
    if (lane == 0) rowb8[row] = make_float2(__fsqrt_ru(s2), __fsqrt_ru(s3));
}

// Per 32-row chunk: {max ||x||, max r8 + (gamma_tc8 + 1.01u) max ||x~8||, P3 (as BF16), beta_min}.
__global__ void __launch_bounds__(256) k1_fp8_stats(const float2 *__restrict__ rowb8, const float4 *__restrict__ cstat,
                                                    int64_t n, int64_t n_pad, float g2, float4 *__restrict__ cstat8)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t chunk = (int64_t)blockIdx.x * 8 + warp;
    if (chunk * 32 >= n_pad) return;
    const int64_t row = chunk * 32 + lane;
    float rq = 0.f, nqt = 0.f;
    if (row < n) {
        const float2 rb = rowb8[row];
        rq = rb.x;
        nqt = rb.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rq = fmaxf(rq, __shfl_xor_sync(0xffffffffu, rq, o));
        nqt = fmaxf(nqt, __shfl_xor_sync(0xffffffffu, nqt, o));
    }
    if (lane == 0) {
        const float4 c = cstat[chunk];
        cstat8[chunk] = make_float4(c.x, __fmaf_ru(g2, nqt, rq), c.z, c.w);
    }
}

int ensure_fp8(Store *s, cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fp8_block) return DL_OK;
    const int dp8 = (s->d + 127) / 128 * 128;
    const size_t b_x = align256((size_t)s->n * dp8), b_sc = align256(sizeof(float) * s->n_pad),
                 b_rb = align256(sizeof(float2) * std::max<int64_t>(s->n, 1)),
                 b_cs = align256(sizeof(float4) * (s->n_pad / 32)), b_scc = align256(sizeof(float) * (s->n_pad / 32));
    void *blk = nullptr;
    int rc = dev_alloc(&blk, b_x + b_sc + b_rb + b_cs + b_scc, st);
    if (rc) return rc;
    char *p = (char *)blk;
    uint8_t *x8 = (uint8_t *)p;
    float *sc8 = (float *)(p + b_x);
    float2 *rowb8 = (float2 *)(p + b_x + b_sc);
    float4 *cstat8 = (float4 *)(p + b_x + b_sc + b_rb);
    float *scc8 = (float *)(p + b_x + b_sc + b_rb + b_cs);
    const unsigned chunk_blocks = (unsigned)((s->n_pad / 32 + 7) / 8);
    if (s->n > 0) {
        k1_fp8_row_scale<<<(unsigned)((s->n + 7) / 8), 256, 0, st>>>(s->x32, s->n, s->d, sc8);
        count_launch();
    }
    k1_fp8_chunk_scale<<<chunk_blocks, 256, 0, st>>>(s->n, s->n_pad, sc8, scc8);
    count_launch();
    if (s->n > 0) {
        k1_fp8<<<(unsigned)((s->n + 7) / 8), 256, 0, st>>>(s->x32, s->n, s->d, dp8, sc8, x8, rowb8);
        count_launch();
    }
    const float g2 = f32_ru(gamma_tc8(dp8) + 1.01 * kU32);
    k1_fp8_stats<<<chunk_blocks, 256, 0, st>>>(rowb8, s->cstat, s->n, s->n_pad, g2, cstat8);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        dev_free(blk, st);
        return cuda_fail(e, "FP8 store copy");
    }
    s->dp8 = dp8;
    s->x8 = x8;
    s->sc8 = sc8;
    s->scc8 = scc8;
    s->rowb8 = rowb8;
    s->cstat8 = cstat8;
    s->fp8_block = blk;
    return DL_OK;
}

// The inner-product join's column term is 0: h = q.x. Its chunk stats come from the same
// kernel as the squared-L2 ones, run on a zero column term, so P1 and P2 (the encoding and
// accumulation terms of the BF16 bound) are the store's own and P3 keeps the L2 beta error
// (a conservative extra); padding rows get +inf, so they never match.
int ensure_ip(Store *s, cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->ip_block) return DL_OK;
    const size_t b_b = align256(sizeof(float) * s->n_pad), b_cs = align256(sizeof(float4) * (s->n_pad / 32));
    void *blk = nullptr;
    int rc = dev_alloc(&blk, b_b + b_cs, st);
    if (rc) return rc;
    float *beta_ip = (float *)blk;
    float4 *cstat_ip = (float4 *)((char *)blk + b_b);
    cudaError_t e = cudaMemsetAsync(beta_ip, 0, sizeof(float) * s->n_pad, st);
    if (e == cudaSuccess) {
        const float g2 = f32_ru(gamma_tc(s->dp) + 1.01 * kU32);
        const float p3a = f32_ru(abs_slack_tc(s->dp));
        k1_chunk_stats<<<(unsigned)((s->n_pad / 32 + 7) / 8), 256, 0, st>>>(beta_ip, s->rowb, s->n, s->n_pad, g2, p3a,
                                                                            beta_ip, cstat_ip);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        dev_free(blk, st);
        return cuda_fail(e, "inner-product column arrays");
    }
    s->beta_ip = beta_ip;
    s->cstat_ip = cstat_ip;
    s->ip_block = blk;
    return DL_OK;
}

// ------------------------------------------------------------------ tensor maps
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

int get_tmap(Store *s, int box_rows, const CUtensorMap **out)
{
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto &t : s->tmaps)
        if (t.valid && t.box_rows == box_rows) {
            *out = &t.map;
            return DL_OK;
        }
    TmapCache *slot = nullptr;
    for (auto &t : s->tmaps)
        if (!t.valid) {
            slot = &t;
            break;
        }
    if (!slot) slot = &s->tmaps[0];
    auto fn = encode_fn();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return DL_ECUDA;
    }
    cuuint64_t gdim[2] = {(cuuint64_t)s->dp, (cuuint64_t)(s->n > 0 ? s->n : 1)};
    cuuint64_t gstride[1] = {(cuuint64_t)s->dp * sizeof(__nv_bfloat16)};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t estride[2] = {1, 1};
    CUresult r = fn(&slot->map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)s->xb, gdim, gstride, box, estride,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d) for dp=%d rows=%lld box=%d", (int)r, s->dp,
                  (long long)s->n, box_rows);
        return DL_ECUDA;
    }
    slot->valid = true;
    slot->box_rows = box_rows;
    *out = &slot->map;
    return DL_OK;
}

int get_tmap8(Store *s, int box_rows, const CUtensorMap **out)
{
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto &t : s->tmaps8)
        if (t.valid && t.box_rows == box_rows) {
            *out = &t.map;
            return DL_OK;
        }
    TmapCache *slot = nullptr;
    for (auto &t : s->tmaps8)
        if (!t.valid) {
            slot = &t;
            break;
        }
    if (!slot) slot = &s->tmaps8[0];
    auto fn = encode_fn();
    if (!fn || !s->x8) {
        set_error("FP8 tensor map: driver entry point or FP8 copy missing");
        return DL_ECUDA;
    }
    cuuint64_t gdim[2] = {(cuuint64_t)s->dp8, (cuuint64_t)(s->n > 0 ? s->n : 1)};
    cuuint64_t gstride[1] = {(cuuint64_t)s->dp8};
    cuuint32_t box[2] = {128, (cuuint32_t)box_rows};
    cuuint32_t estride[2] = {1, 1};
    CUresult r = fn(&slot->map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void *)s->x8, gdim, gstride, box, estride,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled (FP8) failed (%d)", (int)r);
        return DL_ECUDA;
    }
    slot->valid = true;
    slot->box_rows = box_rows;
    *out = &slot->map;
    return DL_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace dl

namespace dl {

// Create a store. With gather == NULL the rows are put in squared-norm order;
// otherwise store row i is caller row gather[i] (device array of n indices).
int store_create_impl(dl_store **out, const int64_t *ids, const float *feats, int64_t n, int32_t d, int32_t where,
                      void *cuda_stream, const int32_t *gather)
{
    clear_error();
    if (!out) {
        set_error("dl_store_create: out is NULL");
        return DL_EINVAL;
    }
    *out = nullptr;
    if (n < 0 || n >= (int64_t(1) << 31)) {
        set_error("dl_store_create: n=%lld out of range [0, 2^31)", (long long)n);
        return DL_EINVAL;
    }
    if (d < 1 || d > 1024) {
        set_error("dl_store_create: d=%d out of range [1, 1024]", d);
        return DL_EINVAL;
    }
    if (n > 0 && (!ids || !feats)) {
        set_error("dl_store_create: ids/feats is NULL");
        return DL_EINVAL;
    }
    if (where != DL_MEM_HOST && where != DL_MEM_DEVICE) {
        set_error("dl_store_create: bad memory kind %d", where);
        return DL_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    dl_store *s = new dl_store();
    s->n = n;
    s->d = d;
    s->dp = (d + 63) / 64 * 64;
    s->n_pad = (n + 255) / 256 * 256;
    if (s->n_pad == 0) s->n_pad = 256;
    DL_CUDA_TRY(cudaGetDevice(&s->device));

    const size_t b_ids = align256(sizeof(int64_t) * n), b_orig = align256(sizeof(int32_t) * n),
                 b_x32 = align256(sizeof(float) * n * d), b_xb = align256(sizeof(__nv_bfloat16) * n * s->dp),
                 b_nq = align256(sizeof(double) * n), b_beta = align256(sizeof(float) * s->n_pad),
                 b_rowb = align256(sizeof(float4) * n), b_cst = align256(sizeof(float4) * (s->n_pad / 32)),
                 b_err = 256;
    const size_t total = b_ids + b_orig + b_x32 + b_xb + b_nq + b_beta + b_rowb + b_cst + b_err;
    void *base = nullptr;
    int rc = dev_alloc(&base, total, st);
    if (rc != DL_OK) {
        delete s;
        return rc;
    }
    char *p = (char *)base;
    s->ids = (int64_t *)p;
    p += b_ids;
    s->orig = (int32_t *)p;
    p += b_orig;
    s->x32 = (float *)p;
    p += b_x32;
    s->xb = (__nv_bfloat16 *)p;
    p += b_xb;
    s->nq64 = (double *)p;
    p += b_nq;
    s->beta = (float *)p;
    p += b_beta;
    s->rowb = (float4 *)p;
    p += b_rowb;
    s->cstat = (float4 *)p;
    p += b_cst;
    int *d_err = (int *)p;

    // scratch for the norm ordering (and for host inputs, the uploaded rows)
    const bool host = (where == DL_MEM_HOST);
    const size_t t_x = host ? align256(sizeof(float) * n * d) : 0, t_ids = host ? align256(sizeof(int64_t) * n) : 0,
                 t_keys = align256(sizeof(float) * n), t_perm = align256(sizeof(int32_t) * n),
                 t_hist = sizeof(unsigned) * kSortBuckets, t_mm = 256;
    void *tmp = nullptr;
    if (n > 0) {
        rc = dev_alloc(&tmp, t_x + t_ids + t_keys + t_perm + t_hist + t_mm, st);
        if (rc != DL_OK) {
            dev_free(base, st);
            delete s;
            return rc;
        }
    }
    auto fail = [&](int code) {
        dev_free(base, st);
        dev_free(tmp, st);
        cudaStreamSynchronize(st);
        delete s;
        return code;
    };
    cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
    if (e != cudaSuccess) return fail(cuda_fail(e, "dl_store_create memset"));
    if (n > 0) {
        char *q = (char *)tmp;
        const float *src_x = feats;
        const int64_t *src_ids = ids;
        if (host) {
            float *hx = (float *)q;
            int64_t *hid = (int64_t *)(q + t_x);
            e = cudaMemcpyAsync(hx, feats, sizeof(float) * n * d, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(hid, ids, sizeof(int64_t) * n, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return fail(cuda_fail(e, "dl_store_create upload"));
            src_x = hx;
            src_ids = hid;
        }
        q += t_x + t_ids;
        float *keys = (float *)q;
        int32_t *perm = (int32_t *)(q + t_keys);
        unsigned *hist = (unsigned *)(q + t_keys + t_perm);
        unsigned *mm = (unsigned *)(q + t_keys + t_perm + t_hist);
        e = cudaMemsetAsync(hist, 0, t_hist, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(mm, 0xff, 4, st);      // min <- 0xffffffff
        if (e == cudaSuccess) e = cudaMemsetAsync(mm + 1, 0, 4, st);     // max <- 0
        if (e != cudaSuccess) return fail(cuda_fail(e, "dl_store_create memset"));
        const unsigned gw = (unsigned)((n + 7) / 8), gt = (unsigned)((n + 255) / 256);
        k_sort_keys<<<gw, 256, 0, st>>>(src_x, n, d, keys, mm);
        if (!gather) {
            k_sort_hist<<<gt, 256, 0, st>>>(keys, n, mm, hist);
            k_sort_scan<<<1, 1024, 0, st>>>(hist);
            k_sort_scatter<<<gt, 256, 0, st>>>(keys, n, mm, hist, perm);
            count_launch(3);
        }
        k_gather_rows<<<gw, 256, 0, st>>>(src_x, src_ids, gather ? gather : perm, n, d, s->x32, s->ids, s->orig);
        k1_norm_quant<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s->x32, n, d, s->dp, s->xb, s->nq64, s->beta,
                                                                  s->rowb, d_err);   // 32 rows per warp
        count_launch(3);
    }
    const float g2 = f32_ru(gamma_tc(s->dp) + 1.01 * kU32);
    const float p3a = f32_ru(abs_slack_tc(s->dp));
    k1_chunk_stats<<<(unsigned)((s->n_pad / 32 + 7) / 8), 256, 0, st>>>(s->beta, s->rowb, n, s->n_pad, g2, p3a, s->beta,
                                                                        s->cstat);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(cuda_fail(e, "store kernels launch"));
    int h_err = 0;
    unsigned h_mm[2] = {0u, 0u};
    if (n > 0) {
        const unsigned *mm = (const unsigned *)((char *)tmp + t_x + t_ids + t_keys + t_perm + t_hist);
        e = cudaMemcpyAsync(h_mm, mm, sizeof h_mm, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return fail(cuda_fail(e, "dl_store_create readback"));
    }
    e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(cuda_fail(e, "dl_store_create sync"));
    if (h_err) {
        set_error("dl_store_create: a feature is non-finite or exceeds 2^40 in magnitude");
        return fail(DL_EINVAL);
    }
    {
        float mx;
        std::memcpy(&mx, &h_mm[1], sizeof mx);
        s->nq_max = mx;
    }
    dev_free(tmp, st);
    *out = s;
    return DL_OK;
}

// ------------------------------------------------------------------ cosine metric
// One warp per store row: the unit-normalized row, written at the caller's row index.
//   n = fl32(sqrt(sum_k x_k^2)), the sum in FP64 with k ascending and each addition
//   rounded to nearest (the products of two floats are exact in FP64); x^_k = fl32(x_k / n).
// A row whose norm is zero has no direction: it is flagged and left zero.
__global__ void __launch_bounds__(256) k_normalize_rows(const float *__restrict__ x32, const int64_t *__restrict__ ids,
                                                        const int32_t *__restrict__ orig, int64_t n, int d,
                                                        float *__restrict__ out, int64_t *__restrict__ out_ids,
                                                        int *__restrict__ err)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * 8 + warp;
    if (row >= n) return;
    const float *xr = x32 + row * d;
    double s = 0.0;
    for (int k0 = 0; k0 < d; k0 += 32) {
        const int k = k0 + lane;
        double sq = 0.0;
        if (k < d) {
            const double v = (double)__ldg(xr + k);
            sq = __dmul_rn(v, v);
        }
        const int lim = min(32, d - k0);
        for (int l = 0; l < lim; ++l) s = __dadd_rn(s, __shfl_sync(0xffffffffu, sq, l));
    }
    const float nr = __double2float_rn(__dsqrt_rn(s));
    const int64_t dst = orig[row];
    float *o = out + dst * d;
    if (!(nr > 0.0f)) {
        for (int k = lane; k < d; k += 32) o[k] = 0.0f;
        if (lane == 0) atomicOr(err, 1);
    } else {
        for (int k = lane; k < d; k += 32) o[k] = __fdiv_rn(__ldg(xr + k), nr);
    }
    if (lane == 0) out_ids[dst] = ids[row];
}

// ------------------------------------------------------------------ chi-square domain
__global__ void __launch_bounds__(256) k_any_negative(const float *__restrict__ x, int64_t n, int *flag)
{
    bool neg = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        neg |= __ldg(x + i) < 0.f;
    if (__any_sync(0xffffffffu, neg) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

int store_nonneg(Store *s, cudaStream_t st, bool *ok)
{
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->nonneg) {
            *ok = s->nonneg == 1;
            return DL_OK;
        }
    }
    const int64_t n = s->n * (int64_t)s->d;
    int h = 0;
    if (n > 0) {
        void *tmp = nullptr;
        int rc = dev_alloc(&tmp, 16, st);
        if (rc) return rc;
        int *flag = (int *)tmp;
        cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
        if (e == cudaSuccess) {
            const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)device_sm_count() * 8);
            k_any_negative<<<grid, 256, 0, st>>>(s->x32, n, flag);
            count_launch();
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        dev_free(tmp, st);
        if (e != cudaSuccess) return cuda_fail(e, "store_nonneg");
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->nonneg = h ? 2 : 1;
    *ok = !h;
    return DL_OK;
}

}  // namespace dl

using namespace dl;

extern "C" {

int dl_store_create(dl_store **out, const int64_t *ids, const float *feats, int64_t n, int32_t d, int32_t where,
                    void *cuda_stream)
{
    dl::NvtxScope nvtx_scope("dl_store_create");
    return store_create_impl(out, ids, feats, n, d, where, cuda_stream, nullptr);
}

int dl_store_normalize(const dl_store *in, dl_store **out, void *cuda_stream)
{
    dl::NvtxScope nvtx_scope("dl_store_normalize");
    clear_error();
    if (!in || !out) {
        set_error("dl_store_normalize: NULL argument");
        return DL_EINVAL;
    }
    *out = nullptr;
    int dev = -1;
    DL_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != in->device) {
        set_error("dl_store_normalize: store lives on device %d but device %d is current", in->device, dev);
        return DL_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int64_t n = in->n;
    const int d = in->d;
    void *tmp = nullptr;
    const size_t b_x = align256(sizeof(float) * (size_t)std::max<int64_t>(n, 1) * d);
    const size_t b_ids = align256(sizeof(int64_t) * (size_t)std::max<int64_t>(n, 1));
    int rc = dev_alloc(&tmp, b_x + b_ids + 256, st);
    if (rc) return rc;
    float *xn = (float *)tmp;
    int64_t *idn = (int64_t *)((char *)tmp + b_x);
    int *d_err = (int *)((char *)tmp + b_x + b_ids);
    cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
    if (e == cudaSuccess && n > 0) {
        k_normalize_rows<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(in->x32, in->ids, in->orig, n, d, xn, idn, d_err);
        count_launch();
        e = cudaGetLastError();
    }
    int h_err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        dev_free(tmp, st);
        return cuda_fail(e, "dl_store_normalize");
    }
    if (h_err) {
        dev_free(tmp, st);
        set_error("dl_store_normalize: a row has a zero norm (no direction for the cosine metric)");
        return DL_EINVAL;
    }
    dl_store *s = nullptr;
    rc = store_create_impl(&s, idn, xn, n, d, DL_MEM_DEVICE, cuda_stream, nullptr);
    cudaStreamSynchronize(st);
    dev_free(tmp, st);
    if (rc) return rc;
    s->unit = true;
    *out = s;
    return DL_OK;
}

int dl_store_destroy(dl_store *s)
{
    if (!s) return DL_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != s->device) cudaSetDevice(s->device);
    dev_free(s->ids, 0);   // ids is the base of the store's single allocation
    if (s->fp8_block) dev_free(s->fp8_block, 0);
    if (s->ip_block) dev_free(s->ip_block, 0);
    if (s->clabel) dev_free(s->clabel, 0);
    for (auto &b : s->balls)
        if (b.blk) dev_free(b.blk, 0);
    if (prev != s->device) cudaSetDevice(prev);
    delete s;
    return DL_OK;
}

int dl_store_shape(const dl_store *s, int64_t *n, int32_t *d)
{
    if (!s) {
        set_error("dl_store_shape: NULL store");
        return DL_EINVAL;
    }
    if (n) *n = s->n;
    if (d) *d = s->d;
    return DL_OK;
}

const char *dl_last_error(void) { return dl::last_error(); }

const char *dl_version(void) { return "dl-simjoin 0.1 (sm_103a)"; }

int64_t dl_kernel_launches(void) { return dl::g_launches.load(); }

}  // extern "C"
