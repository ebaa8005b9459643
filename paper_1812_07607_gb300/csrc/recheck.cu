// recheck.cu -- K6 (exact recheck of band pairs) and the small per-join kernels.
//
// A band pair is one whose low-precision distance could not be placed on one
// side of eps^2 by the error bound. K6 settles it exactly:
//   1. FP32, one warp per pair: D32 = sum_k fl(q_k - x_k)^2 (lane partial FMA
//      chains over 16-byte slices + a shuffle tree), bound |D32 - D| <= (d+8) 2^-24 D
//      + tiny; if that
//      decides the pair against the canonical-FP64 slack, done;
//   2. otherwise a float-float sum (FP32 error-free transformations) whose bound,
//      (d+34)^2 2^-48 D, leaves only near-ties of eps^2 undecided;
//   3. for those, the canonical FP64 value itself: k ascending,
//      t = (double)q_k - (double)x_k, s = s + t*t, every operation rounded to
//      nearest with no contraction (__dsub_rn / __dmul_rn / __dadd_rn), compared
//      with fl64(eps*eps) -- the very expression that defines the result, so the
//      decision is identical to the FP64 nested loop's.
#include <cmath>

#include "checked.cuh"
#include "exact.cuh"
#include "kernels.h"

namespace dl {

__global__ void __launch_bounds__(256)
    k6_recheck(const uint2 *__restrict__ band, const unsigned long long *__restrict__ band_cnt,
               unsigned long long band_cap, const float *__restrict__ R, const float *__restrict__ S, int d, double e2,
               float t_acc, float t_rej, JoinOut out, unsigned long long *__restrict__ n_fp64)
{
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long nb = min(*band_cnt, band_cap);
    const unsigned long long w0 = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    for (unsigned long long i = w0; i < nb; i += nw) {
        const uint2 pr = band[i];
        const bool acc =
            warp_exact_decide(R + (size_t)pr.x * d, S + (size_t)pr.y * d, d, e2, t_acc, t_rej, n_fp64);
        warp_emit(out, acc && lane == 0, false, (int)pr.x, (int)pr.y);
    }
}

// Candidates of the tensor-core kernel -> id pairs. Each warp takes 32 entries:
// proven matches are emitted as they are, the band entries are rechecked by the
// whole warp one after another (vector loads of both rows, FP32 with its bound,
// canonical FP64 if needed), then the warp emits the survivors.
__global__ void __launch_bounds__(256, 5)
    k_finalize(const uint2 *__restrict__ cand, const unsigned long long *__restrict__ cand_cnt,
               unsigned long long cand_cap, const float *__restrict__ R, const float *__restrict__ S, int d, double e2,
               float t_acc, float t_rej, JoinOut out, unsigned long long *__restrict__ n_fp64,
               unsigned long long *__restrict__ n_band, int nR, int nS)
{
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long n = min(*cand_cnt, cand_cap);
    const unsigned long long w0 = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    uint2 nxt = w0 * 32 + lane < n ? cand[w0 * 32 + lane] : make_uint2(0u, 0u);
    for (unsigned long long base = w0 * 32; base < n; base += nw * 32) {
        const unsigned long long i = base + lane;
        const bool valid = i < n;
        uint2 e = nxt;
        nxt = i + nw * 32 < n ? cand[i + nw * 32] : make_uint2(0u, 0u);   // the next window, loaded early
        if (valid && !DL_CHECK(e.x < (unsigned)nR && (e.y & ~kBandFlag) < (unsigned)nS, 20, i)) e = make_uint2(0u, 0u);
        const int r = (int)e.x;
        const int c = (int)(e.y & ~kBandFlag);
        const bool band = valid && (e.y & kBandFlag);
        bool acc = valid && !band;
        bool f64 = false;
        const unsigned bm = __ballot_sync(0xffffffffu, band);
        if (bm) {
            const bool dec = warp_band_decide(bm, R + (size_t)r * d, S + (size_t)c * d, d, e2, t_acc, t_rej, &f64);
            if (band) acc = dec;
        }
        const unsigned fm = __ballot_sync(0xffffffffu, f64);
        if (lane == 0) {
            if (bm) atomicAdd(n_band, (unsigned long long)__popc(bm));
            if (fm) atomicAdd(n_fp64, (unsigned long long)__popc(fm));
        }
        warp_emit(out, acc, false, r, c);
    }
}

// Band pairs of the histogram distances: the canonical FP64 value itself, one pair per
// lane (the band is a relative width of about (d + 10) 2^-22 around eps, so few pairs
// reach it): k ascending, t = (double)q_k - (double)x_k, then s = s + |t| (L1), or
// u = (double)q_k + (double)x_k and, where u > 0, s = s + (t*t)/u (chi-square), every
// operation rounded to nearest with no contraction, compared with eps.
template <int M>
__global__ void __launch_bounds__(256)
    k_hist_recheck(const uint2 *__restrict__ band, const unsigned long long *__restrict__ band_cnt,
                   unsigned long long band_cap, const float *__restrict__ R, const float *__restrict__ S, int d,
                   double eps, JoinOut out, unsigned long long *__restrict__ n_fp64)
{
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long n = min(*band_cnt, band_cap);
    const unsigned long long w0 = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    for (unsigned long long base = w0 * 32; base < n; base += nw * 32) {
        const unsigned long long i = base + lane;
        const bool valid = i < n;
        const uint2 pr = valid ? band[i] : make_uint2(0u, 0u);
        bool acc = false;
        if (valid) {
            const float *q = R + (size_t)pr.x * d, *x = S + (size_t)pr.y * d;
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
            acc = s <= eps;
        }
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        if (lane == 0 && vm) atomicAdd(n_fp64, (unsigned long long)__popc(vm));
        warp_emit(out, acc, false, (int)pr.x, (int)pr.y);
    }
}

// Per-row thresholds of the tensor-core epilogue for one join:
//   alpha_acc = RU32((||q||^2_up - e2 (1 - g64)) / 2)   accept iff h >= alpha_acc + E
//   alpha_rej = RD32((||q||^2_dn - e2 (1 + 2 g64)) / 2) reject iff h <  alpha_rej - E
// with h = q.x - ||x||^2/2 (so D = ||q||^2 - 2h), plus the row's bound terms.
// Padding rows get +inf thresholds (never emit).
__global__ void __launch_bounds__(256)
    k_rowpar(const double *__restrict__ nq64, const float4 *__restrict__ rowb, const float2 *__restrict__ rowb8,
             int64_t n, int64_t n_tot, int dp, double e2_all, const double *__restrict__ row_e2, double g64,
             float4 *__restrict__ rowpar)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_tot) return;
    const float inf = __int_as_float(0x7f800000);
    if (i >= n) {
        rowpar[i] = make_float4(inf, inf, 0.f, 0.f);
        return;
    }
    const double nq = nq64[i];
    const double e2 = row_e2 ? row_e2[i] : e2_all;
    const double rel = (double)(dp + 2) * 2.220446049250313e-16;
    const double nq_up = __dmul_ru(nq, 1.0 + rel);
    const double nq_dn = __dmul_rd(nq, 1.0 - rel);
    const double a_acc = __dsub_ru(nq_up, __dmul_rd(e2, 1.0 - g64)) * 0.5;
    const double a_rej = __dsub_rd(nq_dn, __dmul_ru(e2, 1.0 + 2.0 * g64)) * 0.5;
    const float4 rb = rowb[i];
    const float2 r8 = rowb8 ? rowb8[i] : make_float2(rb.x, rb.y);
    rowpar[i] = make_float4(__double2float_ru(a_acc), __double2float_rd(a_rej), r8.x, r8.y);
}

// Per-row thresholds of the inner-product join (h = q.x, no column term): accept iff
// h >= RU32(t) + E, reject iff h < RD32(t) - E. The row's residual term grows by
// g64 ||q||_up, so that E also covers the canonical dot product's own error,
// |C - q.x| <= g64 sum_k |q_k x_k| <= g64 ||q|| ||x|| (g64 = (dp+4) 2^-53 >= gamma_{d-1}).
__global__ void __launch_bounds__(256)
    k_rowpar_ip(const float4 *__restrict__ rowb, int64_t n, int64_t n_tot, int dp, double t, float4 *__restrict__ rowpar)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_tot) return;
    const float inf = __int_as_float(0x7f800000);
    if (i >= n) {
        rowpar[i] = make_float4(inf, inf, 0.f, 0.f);
        return;
    }
    const float4 rb = rowb[i];   // {||q - q~|| up, ||q~|| up, ||q|| up, beta error}
    const double g64 = (double)(dp + 4) * 1.1102230246251565e-16;
    const float rq = __double2float_ru(__dadd_ru((double)rb.x, __dmul_ru(__dmul_ru((double)rb.z, g64), 1.0 + 0x1p-20)));
    rowpar[i] = make_float4(__double2float_ru(t), __double2float_rd(t), rq, rb.y);
}

// Candidates of the inner-product join -> id pairs: proven matches as they are, band pairs
// decided exactly by warp_band_decide_ip (an FP32 dot with its bound, else the canonical
// FP64 dot); the next window's entries load while this one is decided.
__global__ void __launch_bounds__(256)
    k_finalize_ip(const uint2 *__restrict__ cand, const unsigned long long *__restrict__ cand_cnt,
                  unsigned long long cand_cap, const float *__restrict__ R, const float *__restrict__ S, int d,
                  double t, float t_ru, float t_rd, float cf, float ca, JoinOut out,
                  unsigned long long *__restrict__ n_fp64, unsigned long long *__restrict__ n_band, int nR, int nS)
{
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long n = min(*cand_cnt, cand_cap);
    const unsigned long long w0 = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    uint2 nxt = w0 * 32 + lane < n ? cand[w0 * 32 + lane] : make_uint2(0u, 0u);
    for (unsigned long long base = w0 * 32; base < n; base += nw * 32) {
        const unsigned long long i = base + lane;
        const bool valid = i < n;
        uint2 e = nxt;
        nxt = i + nw * 32 < n ? cand[i + nw * 32] : make_uint2(0u, 0u);
        if (valid && !DL_CHECK(e.x < (unsigned)nR && (e.y & ~kBandFlag) < (unsigned)nS, 21, i)) e = make_uint2(0u, 0u);
        const int r = (int)e.x;
        const int c = (int)(e.y & ~kBandFlag);
        const bool band = valid && (e.y & kBandFlag);
        bool acc = valid && !band;
        bool f64 = false;
        const unsigned bm = __ballot_sync(0xffffffffu, band);
        if (bm) {
            const bool dec =
                warp_band_decide_ip(bm, R + (size_t)r * d, S + (size_t)c * d, d, t, t_ru, t_rd, cf, ca, &f64);
            if (band) acc = dec;
        }
        const unsigned fm = __ballot_sync(0xffffffffu, f64);
        if (lane == 0) {
            if (bm) atomicAdd(n_band, (unsigned long long)__popc(bm));
            if (fm) atomicAdd(n_fp64, (unsigned long long)__popc(fm));
        }
        warp_emit(out, acc, false, r, c);
    }
}

// Self-join full mode: every (i, i) is a pair (canonical D = 0 <= eps^2).
__global__ void __launch_bounds__(256) k_diag(const int64_t *__restrict__ ids, int64_t n, int64_t *out_r,
                                             int64_t *out_s, unsigned long long *out_cnt, unsigned long long cap)
{
    __shared__ unsigned long long base;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t blk0 = (int64_t)blockIdx.x * blockDim.x;
    const int cnt = (int)min((int64_t)blockDim.x, n - blk0);
    if (threadIdx.x == 0) base = atomicAdd(out_cnt, (unsigned long long)cnt);
    __syncthreads();
    if (i < n) {
        const unsigned long long pos = base + threadIdx.x;
        if (pos < cap) {
            out_r[pos] = ids[i];
            out_s[pos] = ids[i];
        }
    }
}

int launch_recheck(const uint2 *band, const unsigned long long *band_cnt, unsigned long long band_cap, const float *R,
                   const float *S, int d, double e2, float t_acc, float t_rej, const JoinOut &out,
                   unsigned long long *n_fp64, int grid, cudaStream_t st)
{
    k6_recheck<<<grid, 256, 0, st>>>(band, band_cnt, band_cap, R, S, d, e2, t_acc, t_rej, out, n_fp64);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k6_recheck launch");
    return DL_OK;
}

int launch_hist_recheck(int metric, const uint2 *band, const unsigned long long *band_cnt, unsigned long long band_cap,
                        const float *R, const float *S, int d, double eps, const JoinOut &out,
                        unsigned long long *n_fp64, int grid, cudaStream_t st)
{
    if (metric == 1)
        k_hist_recheck<1><<<grid, 256, 0, st>>>(band, band_cnt, band_cap, R, S, d, eps, out, n_fp64);
    else
        k_hist_recheck<2><<<grid, 256, 0, st>>>(band, band_cnt, band_cap, R, S, d, eps, out, n_fp64);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_hist_recheck launch");
    return DL_OK;
}

int launch_rowpar_ip(const float4 *rowb, int64_t n, int64_t n_tot, int dp, double t, float4 *rowpar, cudaStream_t st)
{
    if (n_tot <= 0) return DL_OK;
    k_rowpar_ip<<<(unsigned)((n_tot + 255) / 256), 256, 0, st>>>(rowb, n, n_tot, dp, t, rowpar);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_rowpar_ip launch");
    return DL_OK;
}

int launch_finalize_ip(const uint2 *cand, const unsigned long long *cand_cnt, unsigned long long cand_cap,
                       const float *R, const float *S, int d, double t, const JoinOut &out,
                       unsigned long long *n_fp64, unsigned long long *n_band, int grid, cudaStream_t st, int nR, int nS)
{
    // FP32 dot bound: |S32 - q.x| <= (d+2) 2^-24 A, A = sum |q_k x_k| <= A32 (1 + (d+2) 2^-24),
    // plus the canonical dot's (d+4) 2^-53 A; cf = (2d+16) 2^-24 covers both with room, and ca
    // the products that fall below the normal range (at most 2^-149 each).
    const float cf = (float)((2.0 * d + 16.0) * 5.9604644775390625e-08);
    const float ca = (float)((double)d * 1.1210387714598537e-44 + 1.401298464324817e-45);   // d 2^-146 + 2^-149
    float t_ru, t_rd;
    t_ru = (float)t;
    t_rd = (float)t;
    if ((double)t_ru < t) t_ru = std::nextafter(t_ru, __builtin_inff());
    if ((double)t_rd > t) t_rd = std::nextafter(t_rd, -__builtin_inff());
    k_finalize_ip<<<grid, 256, 0, st>>>(cand, cand_cnt, cand_cap, R, S, d, t, t_ru, t_rd, cf, ca, out, n_fp64, n_band, nR,
                                        nS);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_finalize_ip launch");
    return DL_OK;
}

int launch_finalize(const uint2 *cand, const unsigned long long *cand_cnt, unsigned long long cand_cap, const float *R,
                    const float *S, int d, double e2, float t_acc, float t_rej, const JoinOut &out,
                    unsigned long long *n_fp64, unsigned long long *n_band, int grid, cudaStream_t st, int nR, int nS)
{
    k_finalize<<<grid, 256, 0, st>>>(cand, cand_cnt, cand_cap, R, S, d, e2, t_acc, t_rej, out, n_fp64, n_band, nR, nS);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_finalize launch");
    return DL_OK;
}

int launch_rowpar(const double *nq64, const float4 *rowb, int64_t n, int64_t n_tot, int dp, double e2,
                  const double *row_e2, double g64, float4 *rowpar, cudaStream_t st, const float2 *rowb8)
{
    if (n_tot == 0) return DL_OK;
    k_rowpar<<<(unsigned)((n_tot + 255) / 256), 256, 0, st>>>(nq64, rowb, rowb8, n, n_tot, dp, e2, row_e2, g64,
                                                              rowpar);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_rowpar launch");
    return DL_OK;
}

int launch_diag(const int64_t *ids, int64_t n, int64_t *out_r, int64_t *out_s, unsigned long long *out_cnt,
                unsigned long long cap, cudaStream_t st)
{
    if (n == 0) return DL_OK;
    k_diag<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ids, n, out_r, out_s, out_cnt, cap);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_diag launch");
    return DL_OK;
}

}  // namespace dl

DL_CHECK_READER(recheck)
