// join_tc.cu -- K2 + K3 + K5: the tensor-core epsilon-join kernel.
//
// The nested-loop join of Sec. 5 evaluates every pair (q, x). With
//   D(q, x) = ||q||^2 + ||x||^2 - 2 q.x
// the only pair-wise term is the dot product, a dense contraction. This kernel
// computes A = Q~ X~^T on the tcgen05 tensor cores (BF16 in, FP32 accumulate in
// TMEM) and classifies every pair in a fused epilogue against per-row
// thresholds that carry a proven error bound, so that each pair is either a
// proven match, a proven non-match, or an undecided "band" pair that the
// recheck kernel settles exactly.
//
// Per CTA (persistent, one per SM, 192 threads, warp-specialised):
//   warp 0      TMA producer: the 128-row R tile (all d/64 K-chunks) stays
//               resident for a unit; S tiles stream through a ring of stages,
//               one 64-column K-chunk of BN rows per stage (128-byte swizzle).
//   warp 1      MMA issuer: 4 x tcgen05.mma (K=16 each) per stage into one of two
//               TMEM accumulators (128 lanes x BN FP32 columns each), then
//               tcgen05.commit to free the stage / publish the accumulator.
//   warps 2-5   epilogue: tcgen05.ld 32 columns at a time, h = A - beta_x,
//               a running max against the row's reject threshold (2 FP32 ops
//               per pair), and only for the rare chunks that pass, the exact
//               accept/band classification with warp-aggregated output.
// A unit is (R tile m, S tiles [nb, ne)); units are handed out round-robin.
#include <cuda.h>

#include "kernels.h"
#include "ptx.cuh"

namespace dl {



__device__ __forceinline__ bool mbar_wait_plain(uint64_t *bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitBudgetClocks) return false;
    return true;
}

template <int BN>
__global__ void __launch_bounds__(192, 1)
    tc_join_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const TcParams p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int kc = p.kc, stages = p.stages;
    uint8_t *sA = smem;                       // kc x [128 rows x 128 B]
    uint8_t *sB = smem + kc * 16384;          // stages x [BN rows x 128 B]
    uint64_t *bars = reinterpret_cast<uint64_t *>(sB + stages * BN * 128);
    uint64_t *full = bars;                    // [8]
    uint64_t *empty = bars + 8;               // [8]
    uint64_t *a_full = bars + 16;
    uint64_t *a_empty = bars + 17;
    uint64_t *acc_full = bars + 18;           // [2]
    uint64_t *acc_empty = bars + 20;          // [2]
    uint64_t *done = bars + 22;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 24);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 25);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    constexpr uint32_t kTmemCols = 2 * BN;
    constexpr uint32_t kStageBytes = BN * 128;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(a_full, 1);
        mbar_init(a_empty, 1);
        mbar_init(acc_full + 0, 1);
        mbar_init(acc_full + 1, 1);
        mbar_init(acc_empty + 0, 4);
        mbar_init(acc_empty + 1, 4);
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, kTmemCols);
        tmem_relinquish();
    }
    if (warp == 0 && lane == 0) {
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t stage = 0, phase = 0, a_phase = 0;
            uint32_t pend_par[8];
            bool pend[8];
            for (int s = 0; s < 8; ++s) pend[s] = false;
            bool a_pend = false;
            uint32_t a_pend_par = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < p.n_units && ok; u += gridDim.x) {
                const int4 un = p.units[u];
                if (!mbar_wait(a_empty, a_phase ^ 1, abort_flag)) {
                    ok = false;
                    break;
                }
                mbar_arrive_expect_tx(a_full, kc * 16384);
                for (int c = 0; c < kc; ++c) tma_load_2d(sA + c * 16384, &tmA, a_full, c * 64, un.x * 128);
                a_pend = true;
                a_pend_par = a_phase;
                a_phase ^= 1;
                for (int n = un.y; n < un.z && ok; ++n) {
                    for (int c = 0; c < kc; ++c) {
                        if (!mbar_wait(empty + stage, phase ^ 1, abort_flag)) {
                            ok = false;
                            break;
                        }
                        mbar_arrive_expect_tx(full + stage, kStageBytes);
                        tma_load_2d(sB + stage * kStageBytes, &tmB, full + stage, c * 64, n * BN);
                        pend[stage] = true;
                        pend_par[stage] = phase;
                        if (++stage == (uint32_t)stages) {
                            stage = 0;
                            phase ^= 1;
                        }
                    }
                }
            }
            if (!ok) {
                *abort_flag = 1;
                atomicExch(p.err, 1);
                // Let every copy this thread started land before the CTA exits.
                for (int s = 0; s < stages; ++s)
                    if (pend[s]) mbar_wait_plain(full + s, pend_par[s]);
                if (a_pend) mbar_wait_plain(a_full, a_pend_par);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16_f32(128, BN);
            uint32_t stage = 0, phase = 0, a_phase = 0, t = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < p.n_units && ok; u += gridDim.x) {
                const int4 un = p.units[u];
                if (!mbar_wait(a_full, a_phase, abort_flag)) {
                    ok = false;
                    break;
                }
                a_phase ^= 1;
                tc_fence_after();
                for (int n = un.y; n < un.z && ok; ++n) {
                    const uint32_t b = t & 1;
                    if (!mbar_wait(acc_empty + b, ((t >> 1) & 1) ^ 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d_tmem = tmem_base + b * BN;
                    for (int c = 0; c < kc; ++c) {
                        if (!mbar_wait(full + stage, phase, abort_flag)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a_addr = smem_u32(sA + c * 16384);
                        const uint32_t b_addr = smem_u32(sB + stage * kStageBytes);
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            mma_f16(d_tmem, smem_desc_sw128(a_addr + k * 32), smem_desc_sw128(b_addr + k * 32), idesc,
                                    (c | k) != 0);
                        mma_commit(empty + stage);
                        if (++stage == (uint32_t)stages) {
                            stage = 0;
                            phase ^= 1;
                        }
                    }
                    if (!ok) break;
                    mma_commit(acc_full + b);
                    ++t;
                }
                if (ok) mma_commit(a_empty);
            }
            if (!ok) {
                *abort_flag = 1;
                atomicExch(p.err, 1);
            }
            // No MMA may still be running when TMEM is released.
            mma_commit(done);
            mbar_wait_plain(done, 0);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int quad = warp & 3;   // TMEM lanes this warp may access: 32*quad .. +31
        const uint32_t lane_base = static_cast<uint32_t>(quad * 32) << 16;
        uint32_t t = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < p.n_units && ok; u += gridDim.x) {
            const int4 un = p.units[u];
            const int r = un.x * 128 + quad * 32 + lane;
            const float4 rp = p.rowpar[r];
            for (int n = un.y; n < un.z; ++n) {
                const uint32_t b = t & 1;
                if (!mbar_wait(acc_full + b, (t >> 1) & 1, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll 1
                for (int cc = 0; cc < BN / 32; ++cc) {
                    uint32_t v[32];
                    tmem_ld_32x32b_x32(tmem_base + lane_base + b * BN + cc * 32, v);
                    tmem_ld_wait();
                    const int col0 = n * BN + cc * 32;
                    const float4 cs = __ldg(p.cstat + (col0 >> 5));
                    const float eh = __fmaf_ru(rp.z, cs.x, __fmaf_ru(rp.w, cs.y, cs.z));
                    const float tau_rej = __fsub_rd(rp.y, eh);
                    const float4 *b4 = reinterpret_cast<const float4 *>(p.beta + col0);
                    float h[32];
                    float mx = __int_as_float(0xff800000);   // -inf
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float4 bb = __ldg(b4 + i);
                        h[4 * i + 0] = __uint_as_float(v[4 * i + 0]) - bb.x;
                        h[4 * i + 1] = __uint_as_float(v[4 * i + 1]) - bb.y;
                        h[4 * i + 2] = __uint_as_float(v[4 * i + 2]) - bb.z;
                        h[4 * i + 3] = __uint_as_float(v[4 * i + 3]) - bb.w;
                        mx = fmaxf(mx, fmaxf(fmaxf(h[4 * i + 0], h[4 * i + 1]), fmaxf(h[4 * i + 2], h[4 * i + 3])));
                    }
                    if (__any_sync(0xffffffffu, mx >= tau_rej)) {
                        const float tau_acc = __fadd_ru(rp.x, eh);
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int c = col0 + j;
                            const bool valid = (r < p.nR) && (c < p.nS) && (!p.upper || c > r);
                            const bool acc = valid && (h[j] >= tau_acc);
                            const bool band = valid && !acc && (h[j] >= tau_rej);
                            warp_emit(p.out, acc, band, r, c);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acc_empty + b);
                ++t;
            }
        }
        if (!ok) {
            *abort_flag = 1;
            atomicExch(p.err, 1);
        }
    }

    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
    }
}

static size_t tc_smem_bytes(int BN, int kc, int stages)
{
    return 1024 + (size_t)kc * 16384 + (size_t)stages * BN * 128 + 256;
}

int tc_pick_stages(int BN, int kc)
{
    const long avail = 232448 - 1024 - 256 - (long)kc * 16384;
    long s = avail / ((long)BN * 128);
    if (s > 8) s = 8;
    return (int)s;
}



int launch_tc_join(const TcLaunch &L, cudaStream_t st)
{
    const size_t smem = tc_smem_bytes(L.BN, L.p.kc, L.p.stages);
    cudaError_t e;
    if (L.BN == 256) {
        e = cudaFuncSetAttribute(tc_join_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(tc_join_kernel<256>)");
        tc_join_kernel<256><<<L.grid, 192, smem, st>>>(*L.tmA, *L.tmB, L.p);
    } else if (L.BN == 128) {
        e = cudaFuncSetAttribute(tc_join_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(tc_join_kernel<128>)");
        tc_join_kernel<128><<<L.grid, 192, smem, st>>>(*L.tmA, *L.tmB, L.p);
    } else {
        set_error("tensor-core tile width %d not supported (128 or 256)", L.BN);
        return DL_EINVAL;
    }
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tc_join_kernel launch");
    return DL_OK;
}

}  // namespace dl
