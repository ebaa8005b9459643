// join_simt.cu -- K8: the FP32 SIMT join (plain baseline and exact-path front end).
//
// The nested-loop join of Sec. 5 evaluated directly as D32 = sum_k fl(q_k - x_k)^2
// with an FMA chain per pair, register-tiled 8x8 pairs per thread over a
// 128 x 128 pair tile staged through shared memory in 32-wide K slices. The same
// tiling evaluates the histogram distances (L1, chi-square), which are not
// contractions and so stay on the CUDA cores; their thresholds carry their own
// FP32 bounds and their band pairs go to k_hist_recheck.
//
//   plain (DL_PREC_FP32_PLAIN): accept iff D32 <= fl32(eps)^2 -- the usual FP32
//     GPU join, the throughput baseline; not exact near the threshold.
//   exact (DL_PREC_FP32): accept iff D32 <= t_acc, reject iff D32 > t_rej, where
//     the thresholds carry the FP32 error bound |D32 - D| <= (d+8) 2^-24 D plus
//     the canonical-FP64 slack; undecided pairs go to the recheck (K6).
#include "kernels.h"

namespace dl {

constexpr int kSimtTile = 128;
constexpr int kSimtK = 32;



__device__ __forceinline__ long long tri_start(int m, int T) { return (long long)m * T - (long long)m * (m - 1) / 2; }

// One distance term of metric M for the pair (a, b) of feature values, added to acc:
//   M = 0: squared L2, acc += (a - b)^2 (one FMA);
//   M = 1: L1, acc += |a - b|;
//   M = 2: chi-square on non-negative features, acc += (a - b)^2 / (a + b) with the
//          reciprocal from rcp.approx (relative error <= 2^-23), 0 when a + b is 0 or
//          subnormal (then the exact term is at most a + b < 2^-126).
template <int M>
__device__ __forceinline__ void dist_term(float a, float b, float &acc)
{
    const float t = a - b;
    if constexpr (M == 0) {
        acc = fmaf(t, t, acc);
    } else if constexpr (M == 1) {
        acc += fabsf(t);
    } else {
        const float u = a + b;
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(u));
        const float term = (t * t) * r;
        acc += (u >= 1.17549435e-38f) ? term : 0.f;
    }
}

template <int M>
__global__ void __launch_bounds__(256) k8_simt_join(const SimtParams p)
{
    __shared__ __align__(16) float As[kSimtK][kSimtTile + 4];
    __shared__ __align__(16) float Bs[kSimtK][kSimtTile + 4];

    int tm, tn;
    if (p.upper) {
        const int T = p.tiles_m;
        const long long l = blockIdx.x;
        const double tt = 2.0 * T + 1.0;
        int m = (int)floor((tt - sqrt(tt * tt - 8.0 * (double)l)) * 0.5);
        if (m < 0) m = 0;
        if (m > T - 1) m = T - 1;
        while (m > 0 && tri_start(m, T) > l) --m;
        while (m + 1 < T && tri_start(m + 1, T) <= l) ++m;
        tm = m;
        tn = m + (int)(l - tri_start(m, T));
    } else {
        tm = blockIdx.y;
        tn = blockIdx.x;
    }
    const int r0 = tm * kSimtTile, c0 = tn * kSimtTile;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    for (int k0 = 0; k0 < p.d; k0 += kSimtK) {
        // stage a 128-row x 32-column slice of each operand, transposed to [k][row]
#pragma unroll 4
        for (int i = 0; i < 16; ++i) {
            const int e = tid + 256 * i;
            const int row = e >> 5, k = e & 31;
            const int gk = k0 + k;
            const int gr = r0 + row, gc = c0 + row;
            As[k][row] = (gr < p.nR && gk < p.d) ? __ldg(p.R + (size_t)gr * p.d + gk) : 0.f;
            Bs[k][row] = (gc < p.nS && gk < p.d) ? __ldg(p.S + (size_t)gc * p.d + gk) : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < kSimtK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[k][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[k][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) dist_term<M>(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }

    // classify: the common case is "no candidate anywhere in this thread's 64 pairs"
    bool any = false;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) any |= (p.exact ? (acc[i][j] <= p.t_rej) : (acc[i][j] <= p.t_acc));
    if (!__any_sync(0xffffffffu, any)) return;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = r0 + ((i < 4) ? (ty * 4 + i) : (64 + ty * 4 + i - 4));
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = c0 + ((j < 4) ? (tx * 4 + j) : (64 + tx * 4 + j - 4));
            const bool valid = (r < p.nR) && (c < p.nS) && (!p.upper || c > r);
            const float v = acc[i][j];
            const bool a = valid && (v <= p.t_acc);
            const bool b = valid && p.exact && !a && (v <= p.t_rej);
            warp_emit(p.out, a, b, r, c);
        }
    }
}



int launch_simt_join(SimtParams p, cudaStream_t st)
{
    const int tm = (p.nR + kSimtTile - 1) / kSimtTile;
    const int tn = (p.nS + kSimtTile - 1) / kSimtTile;
    p.tiles_m = tm;
    if (tm == 0 || tn == 0) return DL_OK;
    if (p.upper) {
        const long long blocks = (long long)tm * (tm + 1) / 2;
        if (blocks > 2147483647LL) {
            set_error("self-join too large for the SIMT path");
            return DL_EUNSUPPORTED;
        }
        if (p.metric == 1) k8_simt_join<1><<<(unsigned)blocks, 256, 0, st>>>(p);
        else if (p.metric == 2) k8_simt_join<2><<<(unsigned)blocks, 256, 0, st>>>(p);
        else k8_simt_join<0><<<(unsigned)blocks, 256, 0, st>>>(p);
    } else {
        if (tm > 65535) {
            set_error("R too large for the SIMT path grid");
            return DL_EUNSUPPORTED;
        }
        const dim3 grid((unsigned)tn, (unsigned)tm);
        if (p.metric == 1) k8_simt_join<1><<<grid, 256, 0, st>>>(p);
        else if (p.metric == 2) k8_simt_join<2><<<grid, 256, 0, st>>>(p);
        else k8_simt_join<0><<<grid, 256, 0, st>>>(p);
    }
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k8_simt_join launch");
    return DL_OK;
}

}  // namespace dl
