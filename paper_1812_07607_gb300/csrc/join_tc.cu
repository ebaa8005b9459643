// join_tc.cu -- K2 + K3 + K5: the tensor-core epsilon-join kernel.
//
// The nested-loop join of Sec. 5 evaluates every pair (q, x). With
//   D(q, x) = ||q||^2 + ||x||^2 - 2 q.x
// the only pair-wise term is the dot product, a dense contraction. This kernel
// computes A = Q~ X~^T on the tcgen05 tensor cores (BF16 or FP8 e4m3 in, FP32
// accumulate in TMEM) and classifies every pair in a fused epilogue against per-row
// thresholds that carry a proven error bound, so that each pair is either a proven
// match, a proven non-match, or an undecided "band" pair that the recheck settles
// exactly. With h = q.x - ||x||^2/2 the epilogue works on h~ = fl(A s - beta)
// (s = 1 for BF16; for FP8 the exact power of two s_q s_chunk).
//
// Per CTA (persistent, one per SM, 320 threads, warp-specialised):
//   warp 0      TMA producer: the 128-row R tile (all K chunks of 128 bytes: 64 BF16
//               or 128 FP8 columns) is loaded once per unit into one of one or two A
//               slots; S tiles stream through a ring of stages, one K chunk of BN
//               rows per stage (128-byte swizzle).
//   warp 1      MMA issuer: 4 x tcgen05.mma (K = 32 bytes each) per stage into one of
//               the 512 / BN TMEM accumulators (128 lanes x BN FP32 columns each: two
//               of 256 or four of 128 columns), then tcgen05.commit to free the stage
//               and to publish the accumulator.
//   warps 2-9   epilogue, two warps per TMEM lane quadrant, each owning half of the
//               tile's columns. Per 64-column piece: tcgen05.ld, then a three-input max
//               tree over the raw accumulators of each 32-column chunk and one compare
//               of fl_ru(max A * s - beta_min of the chunk) against the row's reject
//               threshold (about half an issue slot per pair; store rows are in norm
//               order so a chunk's betas are nearly equal). Only chunks that this
//               bound cannot reject are classified pair by pair (slow_chunk): proven
//               matches and band pairs go to a per-warp shared-memory buffer as (r, c)
//               candidates, flushed to the global candidate list with one atomic per
//               flush. The column data (beta, chunk stats, FP8 chunk scales) of the
//               next tile is staged with cp.async while the current one is processed.
//               k_finalize turns the candidates into id pairs.
// A unit is (R tile m, S tiles [nb, ne)); units are handed out round-robin, in the
// S-range-major order their builders produce.
#include <algorithm>
#include <atomic>

#include <cuda.h>

#include "kernels.h"
#include "checked.cuh"
#include "ptx.cuh"

namespace dl {

__device__ __forceinline__ bool mbar_wait_plain(uint64_t *bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitBudgetClocks) return false;
    return true;
}

// The S tile after n in a unit of R tile m ending at `end`: n + 1, or with a tile mask the
// next tile whose bit is set (end when there is none). Every role steps through a unit with
// it, so all of them see the same tile sequence.
template <bool MASK>
__device__ __forceinline__ int tile_after(const TcParams &p, int m, int n, int end)
{
    ++n;
    if constexpr (MASK) {
        const uint32_t *row = p.tile_mask + (size_t)m * p.mask_ntw;
        while (n < end) {
            const uint32_t w = __ldg(row + (n >> 5)) >> (n & 31);
            if (w) return min(n + __ffs((int)w) - 1, end);
            n = (n | 31) + 1;
        }
        return end;
    }
    return n;
}

// Walks this CTA's (unit, S tile) sequence.
template <bool MASK>
struct TileIter {
    int u, n;
    int4 un;
    bool valid;
    int stride;
    int nu;   // unit count
    __device__ __forceinline__ void start(const TcParams &p, int first, int step, int n_units)
    {
        u = first;
        stride = step;
        nu = n_units;
        valid = u < nu;
        if (valid) {
            un = p.units[u];
            n = un.y;
        }
    }
    __device__ __forceinline__ void next(const TcParams &p)
    {
        if (!valid) return;
        n = tile_after<MASK>(p, un.x, n, un.z);
        if (n == un.z) {
            u += stride;
            valid = u < nu;
            if (valid) {
                un = p.units[u];
                n = un.y;
            }
        }
    }
};

constexpr int kStageCap = 128;   // candidate entries a warp buffers before flushing
// Epilogue warps: 8 (each owning BN/2 columns of a tile, loaded 64 at a time), or -- the wide
// epilogue of the epsilon-join on 256-column tiles -- 16 (four per SM sub-partition, 64 columns
// each, loaded 32 at a time), which keeps up better when many chunks hold candidates.
__host__ __device__ constexpr int tc_epi_warps(bool wide) { return wide ? 16 : 8; }
__host__ __device__ constexpr int tc_threads(bool wide) { return 64 + 32 * tc_epi_warps(wide); }
constexpr int kColSlots = 2;     // epilogue column-data slots: the current tile and the next

// Copy a warp's buffered candidates to the global list (one atomic per flush).
__device__ __forceinline__ void flush_stage(const TcParams &p, uint2 *stg, uint32_t &scnt)
{
    const unsigned lane = threadIdx.x & 31;
    __syncwarp();
    unsigned long long base = 0;
    if (lane == 0 && scnt) base = atomicAdd(p.cand_cnt, (unsigned long long)scnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (uint32_t i = lane; i < scnt; i += 32) {
        const unsigned long long idx = base + i;
        if (idx < p.cand_cap) p.cand[idx] = stg[i];
    }
    __syncwarp();
    scnt = 0;
}

// Pair-by-pair path for one 32-column chunk, for pairs (r, c0 + j) with h = fl(A s - beta_j)
// (s = 1 for BF16; for FP8 the exact power of two s_q s_chunk, so one rounding). A pair with
// h >= tau_rej of its row -- a proven match
// (h >= tau_acc) or a band pair -- becomes a candidate. Warp-collective; `hit` marks the
// lanes (rows) whose chunk bound failed, the others have no candidate in this chunk.
//  * Few such rows: they are taken one at a time, the row's 32 values passing through the
//    warp's shared-memory exchange slot so that lane j classifies column c0 + j; the
//    candidates' buffer positions come from a ballot prefix.
//  * Many such rows: every lane classifies its own row's 32 columns into a bit mask, a
//    warp prefix sum of the mask counts places each lane's candidates.
template <bool FP8, int N>
__device__ __forceinline__ uint32_t slow_chunk(const TcParams &p, const uint32_t (&v)[N], int o, const float *bt,
                                               float sc, float tau_acc, float tau_rej, bool hit, int r, int c0,
                                               float *xch, uint2 *stg, uint32_t scnt)
{
    const unsigned lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    unsigned hm = __ballot_sync(0xffffffffu, hit);
    if (__popc(hm) > 3) {
        uint32_t cm = 0, am = 0;
        if (hit) {
            const float4 *bt4 = reinterpret_cast<const float4 *>(bt + o);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float4 b4 = bt4[q];
                const float bq[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int j = 4 * q + i;
                    const float h = __fmaf_rn(__uint_as_float(v[o + j]), sc, -bq[i]);
                    cm |= (h >= tau_rej ? 1u : 0u) << j;
                    am |= (h >= tau_acc ? 1u : 0u) << j;
                }
            }
            const int rem = p.nS - c0;   // columns past the store
            if (rem < 32) cm &= rem <= 0 ? 0u : ((1u << rem) - 1u);
            if (p.upper) {   // upper mode: only pairs with c > r
                const int k = r - c0;
                if (k >= 31)
                    cm = 0u;
                else if (k >= 0)
                    cm &= ~((2u << k) - 1u);
            }
        }
        const uint32_t nl = __popc(cm);
        uint32_t incl = nl;
#pragma unroll
        for (int sft = 1; sft < 32; sft <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, sft);
            if ((int)lane >= sft) incl += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        if (total == 0) return scnt;
        uint2 *dst;
        unsigned long long lim;
        if (total <= (uint32_t)kStageCap) {
            if (scnt + total > (uint32_t)kStageCap) flush_stage(p, stg, scnt);
            dst = stg + scnt;
            lim = ~0ULL;
            scnt += total;
        } else {   // more than a buffer: reserve the space in the global list directly
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(p.cand_cnt, (unsigned long long)total);
            base = __shfl_sync(0xffffffffu, base, 0);
            dst = p.cand + base;
            lim = base < p.cand_cap ? p.cand_cap - base : 0ULL;
        }
        unsigned long long k = incl - nl;
        while (cm) {
            const int j = __ffs(cm) - 1;
            cm &= cm - 1u;
            // staged (lim = ~0) entries must stay inside the warp's kStageCap buffer
            if (k < lim && DL_CHECK(lim != ~0ULL || k < (unsigned long long)kStageCap, 1, k))
                dst[k] = make_uint2((uint32_t)r, (uint32_t)(c0 + j) | (((am >> j) & 1u) ? 0u : kBandFlag));
            ++k;
        }
        return scnt;
    }
    const int c = c0 + (int)lane;                        // this lane's column
    const float bl = bt[o + lane];
    const bool cvalid = c < p.nS;
    while (hm) {
        const int k = __ffs(hm) - 1;
        hm &= hm - 1u;
        if ((int)lane == k) {
            float4 *x4 = reinterpret_cast<float4 *>(xch);
#pragma unroll
            for (int i = 0; i < 8; ++i)
                x4[i] = make_float4(__uint_as_float(v[o + 4 * i]), __uint_as_float(v[o + 4 * i + 1]),
                                    __uint_as_float(v[o + 4 * i + 2]), __uint_as_float(v[o + 4 * i + 3]));
        }
        __syncwarp();
        const float a = xch[lane];
        __syncwarp();   // every lane has read the slot before the next row overwrites it
        const float h = __fmaf_rn(a, __shfl_sync(0xffffffffu, sc, k), -bl);
        const float ta = __shfl_sync(0xffffffffu, tau_acc, k);
        const float tr = __shfl_sync(0xffffffffu, tau_rej, k);
        const int rk = __shfl_sync(0xffffffffu, r, k);
        const bool cand = cvalid && h >= tr && (!p.upper || c > rk);   // upper mode: pairs with c > r only
        const unsigned cm = __ballot_sync(0xffffffffu, cand);
        if (cm) {
            if (scnt + __popc(cm) > (uint32_t)kStageCap) flush_stage(p, stg, scnt);
            if (cand && DL_CHECK(scnt + __popc(cm & lt) < (uint32_t)kStageCap, 2, scnt + __popc(cm & lt)))
                stg[scnt + __popc(cm & lt)] = make_uint2((uint32_t)rk, (uint32_t)c | (h >= ta ? 0u : kBandFlag));
            scnt += __popc(cm);
        }
    }
    return scnt;
}

// ---------------------------------------------------------------- top-k epilogue
constexpr int kHeapArity = 8;   // children per node of a top-k slot's heap (8 measured faster than 4 and 2)

// A slot's state is (theta, list fill) in registers plus, in global memory, a kHeapArity-ary
// min-heap of the k largest lower bounds L = fl_rd(h - E) seen so far above the row's
// published threshold (theta is its minimum: at least k columns have h >= theta) and
// the list of every column
// whose upper bound U = fl_ru(h + E) reached theta when it was seen. Every true
// top-k column has U >= h >= the k-th largest h >= theta, so it is in the list.
// Returns the new (theta, fill) packed in a float2.
__device__ __noinline__ float2 topk_insert(const TcParams &p, size_t sidx, int r, int c, float U, float L,
                                           float theta, int cnt, float theta_row)
{
    uint2 *list = p.tk_list + sidx * (size_t)p.tk_cap;
    if (cnt >= p.tk_cap) {   // compact: drop columns whose upper bound fell below the best threshold
        const float th = fmaxf(theta, float_from_order_code(__ldcg(p.tk_row_theta + r)));
        int w = 0;
        for (int i = 0; i < cnt; ++i) {
            const uint2 e = list[i];
            if (__uint_as_float(e.y) >= th) list[w++] = e;
        }
        cnt = w;
        if (cnt >= p.tk_cap) {
            p.tk_overflow[r] = 1;   // the exact fallback re-solves this row
            return make_float2(theta, __int_as_float(cnt));
        }
    }
    list[cnt++] = make_uint2((uint32_t)c, __float_as_uint(U));
    // The heap only needs lower bounds above every threshold already known for the row: a
    // bound at or below the row's threshold can raise neither this slot's threshold past it
    // nor the k-th largest bound that finalize takes over all heaps (which stays <= the
    // row's k-th largest h either way), so it is not inserted.
    if (L > fmaxf(theta, theta_row)) {
        float *heap = p.tk_heap + sidx * (size_t)p.tk_k;
        const int k = p.tk_k;
        int i = 0;
        // replace the minimum by L and sift down a kHeapArity-ary heap (children of i at
        // kHeapArity * i + 1 ...): a third of a binary heap's levels at k = 100, the loads of
        // a level issued together
        while (true) {
            const int c0 = kHeapArity * i + 1;
            if (c0 >= k) break;
            float hc[kHeapArity];
#pragma unroll
            for (int j = 0; j < kHeapArity; ++j) hc[j] = c0 + j < k ? heap[c0 + j] : __int_as_float(0x7f800000);
            int m = c0;
            float hm = hc[0];
#pragma unroll
            for (int j = 1; j < kHeapArity; ++j)
                if (hc[j] < hm) {
                    hm = hc[j];
                    m = c0 + j;
                }
            if (hm >= L) break;
            heap[i] = hm;
            i = m;
        }
        heap[i] = L;
        theta = heap[0];
        atomicMax(p.tk_row_theta + r, float_order_code(theta));   // share with the row's other slots
    }
    return make_float2(theta, __int_as_float(cnt));
}

// Top-k slow path for a 64-column piece some lane could not reject: each lane
// walks its own row's columns whose upper bound reaches its theta.
__device__ __forceinline__ void slow_topk(const TcParams &p, const uint32_t (&v)[64], const float *bt, float eh0,
                                          float eh1, bool hit0, bool hit1, int r, int col0, size_t sidx,
                                          float &theta, int &cnt, float theta_row)
{
    if (r >= p.nR) return;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
        if (!(hh ? hit1 : hit0)) continue;
        const float eh = hh ? eh1 : eh0;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int c = col0 + hh * 32 + j;
            const float h = __uint_as_float(v[hh * 32 + j]) - bt[hh * 32 + j];
            const float U = __fadd_ru(h, eh);
            if (c < p.nS && U >= fmaxf(theta, theta_row)) {
                const float2 st = topk_insert(p, sidx, r, c, U, __fsub_rd(h, eh), theta, cnt, theta_row);
                theta = st.x;
                cnt = __float_as_int(st.y);
            }
        }
    }
}

// Maximum of v[o .. o+31] with three-input max.f32 (17 instructions, depth 4).
__device__ __forceinline__ float fmax3(float a, float b, float c)
{
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

template <int N>
__device__ __forceinline__ float max_tree32(const uint32_t (&v)[N], int o)
{
    float m[11];
#pragma unroll
    for (int i = 0; i < 10; ++i)
        m[i] = fmax3(__uint_as_float(v[o + 3 * i]), __uint_as_float(v[o + 3 * i + 1]), __uint_as_float(v[o + 3 * i + 2]));
    m[10] = fmaxf(__uint_as_float(v[o + 30]), __uint_as_float(v[o + 31]));
    const float a = fmax3(m[0], m[1], m[2]), b = fmax3(m[3], m[4], m[5]), c = fmax3(m[6], m[7], m[8]);
    const float e = fmaxf(m[9], m[10]);
    return fmaxf(fmax3(a, b, c), e);
}

// CG2: a CTA pair (cluster of two) computes 256-row tiles with tcgen05 cta_group::2. Each
// CTA loads its own 128 rows of A and its own half (BN/2 rows) of every S tile into its own
// shared memory, signalling its own barriers; the peer CTA's otherwise idle MMA warp forwards
// each of its completions to the leader (rank 0), whose single thread issues M = 256 MMAs that
// read both CTAs' operands and write each CTA's 128 rows into that CTA's TMEM; commits are
// multicast to both CTAs. Each CTA's epilogue handles its own rows; the peer releases an
// accumulator with a remote arrive on the leader's barrier. Half the B bytes per stage means
// twice the stages in the same shared memory beside a resident R tile.
template <int BN, bool TOPK, bool FP8, bool CG2, bool WIDE, bool MASK, bool STREAM>
__global__ void __launch_bounds__(tc_threads(WIDE), 1)
    tc_join_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const TcParams p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int kc = p.kc, stages = p.stages, a_slots = p.a_slots;
    constexpr uint32_t kStageBytes = (CG2 ? BN / 2 : BN) * 128;   // this CTA's rows of an S tile x 128 B
    // STREAM: no resident R tile; each stage also carries the R tile's matching 128-byte K chunk
    // (128 rows, 16 KB), so a large d keeps four stages instead of two beside a resident tile
    static_assert(!STREAM || (!CG2 && !TOPK && !MASK), "streamed R chunks serve the one-SM epsilon-join");
    constexpr uint32_t kStageStride = STREAM ? kStageBytes + 16384 : kStageBytes;
    constexpr int kChunkCols = FP8 ? 128 : 64;   // columns per 128-byte K chunk
    constexpr int kAcc = 512 / BN;              // TMEM accumulators: 2 of 256 or 4 of 128 columns
    constexpr uint32_t kTmemCols = 512;
    static_assert(!WIDE || BN == 256, "the wide epilogue serves 256-column tiles");
    constexpr int kEpi = tc_epi_warps(WIDE);   // epilogue warps
    constexpr int HC = BN * 4 / kEpi;        // columns of a tile each epilogue warp owns (128 or 64)
    constexpr int kSubW = HC / 32;           // 32-column chunks per warp per tile
    const uint32_t a_bytes = (uint32_t)kc * 16384;
    uint8_t *sA = smem;                                    // a_slots x kc x [128 rows x 128 B]
    uint8_t *sB = smem + (STREAM ? 0 : a_slots * a_bytes);   // stages x [BN rows x 128 B (+ R chunk)]
    // Column data of a tile (beta, chunk stats, FP8 chunk scales) is staged by the epilogue
    // warps themselves with cp.async, one tile ahead, in kColSlots = 2 slots.
    float *s_beta = reinterpret_cast<float *>(sB + stages * kStageStride);    // kEpi warps x kColSlots x HC: beta
    float4 *s_cst = reinterpret_cast<float4 *>(s_beta + kEpi * kColSlots * HC); // kEpi x kColSlots x kSubW chunk stats
    uint2 *s_stage = reinterpret_cast<uint2 *>(s_cst + kEpi * kColSlots * kSubW);   // kEpi x kStageCap candidates
    float *s_sx = reinterpret_cast<float *>(s_stage + kEpi * kStageCap);     // FP8: kEpi x kColSlots x kSubW scales
    uint64_t *bars = reinterpret_cast<uint64_t *>(s_sx + (FP8 ? kEpi * kColSlots * kSubW : 0));
    uint64_t *full = bars;                    // [8]
    uint64_t *empty = bars + 8;               // [8]
    uint64_t *a_full = bars + 16;             // [2]
    uint64_t *a_empty = bars + 18;            // [2]
    uint64_t *acc_full = bars + 20;           // [kAcc <= 4]
    uint64_t *acc_empty = bars + 24;          // [kAcc <= 4]
    uint64_t *done = bars + 28;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 29);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 30);
    uint64_t *pfull = bars + 32;              // CG2 leader: [8] the peer's half of the stage landed
    uint64_t *pa_full = bars + 40;            // CG2 leader: [2] the peer's rows of the R tile landed
    float *s_xch = reinterpret_cast<float *>(bars + 48);   // [kEpi warps x 32] row exchange slots (16-byte aligned)

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t crank = CG2 ? cluster_ctarank() : 0u;   // this CTA's rank in its pair
    const bool leader = crank == 0u;
    const int ufirst = CG2 ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;   // units are per CTA pair with CG2
    const int ustride = CG2 ? (int)(gridDim.x >> 1) : (int)gridDim.x;
    const int n_units = MASK ? *p.n_units_dev : p.n_units;   // MASK: units built on the device
    constexpr int kRowTiles = CG2 ? 2 : 1;    // 128-row tiles per unit row tile
    // Raise the abort flag of this CTA (and of the peer, so that it stops waiting too).
    auto raise_abort = [&]() {
        *abort_flag = 1;
        if constexpr (CG2) st_shared_remote_u32(mapa_shared(const_cast<int *>(abort_flag), crank ^ 1u), 1u);
        atomicExch(p.err, 1);
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(a_full + s, 1);
            mbar_init(a_empty + s, 1);
        }
        for (int s = 0; s < kAcc; ++s) {
            mbar_init(acc_full + s, 1);
            mbar_init(acc_empty + s, CG2 ? 2 * kEpi : kEpi);   // CG2 (leader): both CTAs' epilogue warps
        }
        if constexpr (CG2) {
            for (int s = 0; s < 8; ++s) mbar_init(pfull + s, 1);
            for (int s = 0; s < 2; ++s) mbar_init(pa_full + s, 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc<CG2>(tmem_slot, kTmemCols);
        tmem_relinquish<CG2>();
    }
    if (warp == 0 && lane == 0) {
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
    }
    tc_fence_before();
    __syncthreads();
    if constexpr (CG2) cluster_sync_all();   // both CTAs' barriers initialised and TMEM allocated
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t stage = 0, phase = 0;
            uint32_t pend_par[8], a_pend_par[2];
            bool pend[8], a_pend[2] = {false, false};
            for (int s = 0; s < 8; ++s) pend[s] = false;
            bool ok = true;
            int i = 0;   // unit count of this CTA
            for (int u = ufirst; u < n_units && ok; u += ustride, ++i) {
                const int4 un = p.units[u];
                if constexpr (!STREAM) {
                    const int slot = i % a_slots;
                    const uint32_t use = (uint32_t)(i / a_slots);
                    if (!mbar_wait(a_empty + slot, (use & 1) ^ 1, abort_flag, p.wait_budget)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(a_full + slot, a_bytes);
                    for (int c = 0; c < kc; ++c)   // a K chunk is 128 bytes: 64 BF16 or 128 FP8 columns
                        tma_load_2d(sA + slot * a_bytes + c * 16384, &tmA, a_full + slot, c * kChunkCols,
                                    (un.x * kRowTiles + (int)crank) * 128);
                    a_pend[slot] = true;
                    a_pend_par[slot] = use & 1;
                }
                for (int n = un.y; n < un.z && ok; n = tile_after<MASK>(p, un.x, n, un.z)) {
                    for (int c = 0; c < kc; ++c) {
                        if (!mbar_wait(empty + stage, phase ^ 1, abort_flag, p.wait_budget)) {
                            ok = false;
                            break;
                        }
                        mbar_arrive_expect_tx(full + stage, kStageStride);
                        tma_load_2d(sB + stage * kStageStride, &tmB, full + stage, c * kChunkCols,
                                    n * BN + (CG2 ? (int)crank * (BN / 2) : 0));
                        if constexpr (STREAM)   // the R tile's chunk c beside it
                            tma_load_2d(sB + stage * kStageStride + kStageBytes, &tmA, full + stage, c * kChunkCols,
                                        un.x * 128);
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
                raise_abort();
                // Let every copy this thread started land before the CTA exits.
                for (int s = 0; s < stages; ++s)
                    if (pend[s]) mbar_wait_plain(full + s, pend_par[s]);
                for (int s = 0; s < 2; ++s)
                    if (a_pend[s]) mbar_wait_plain(a_full + s, a_pend_par[s]);
            }
        }
    } else if (warp == 1 && CG2 && !leader) {
        // ------------------------------------------------------------ peer: completion forwarder
        // The leader's MMAs read this CTA's shared memory too: forward each completion of this
        // CTA's own R-tile and stage barriers, in the producer's order, to the leader.
        if (lane == 0) {
            const uint32_t r_pfull = mapa_shared(pfull, 0u), r_pa_full = mapa_shared(pa_full, 0u);
            uint32_t stage = 0, phase = 0;
            bool ok = true;
            int i = 0;
            for (int u = ufirst; u < n_units && ok; u += ustride, ++i) {
                const int4 un = p.units[u];
                const int slot = i % a_slots;
                const uint32_t use = (uint32_t)(i / a_slots);
                if (!mbar_wait(a_full + slot, use & 1, abort_flag, p.wait_budget)) {
                    ok = false;
                    break;
                }
                mbar_arrive_remote(r_pa_full + (uint32_t)slot * 8u);
                for (int n = un.y; n < un.z && ok; n = tile_after<MASK>(p, un.x, n, un.z)) {
                    for (int c = 0; c < kc; ++c) {
                        if (!mbar_wait(full + stage, phase, abort_flag, p.wait_budget)) {
                            ok = false;
                            break;
                        }
                        mbar_arrive_remote(r_pfull + stage * 8u);
                        if (++stage == (uint32_t)stages) {
                            stage = 0;
                            phase ^= 1;
                        }
                    }
                }
            }
            if (!ok) raise_abort();
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc =
                FP8 ? idesc_e4m3_f32(CG2 ? 256 : 128, BN) : idesc_bf16_f32(CG2 ? 256 : 128, BN);
            uint32_t stage = 0, phase = 0, t = 0;
            bool ok = true, any_mma = false;
            int i = 0;
            for (int u = ufirst; u < n_units && ok; u += ustride, ++i) {
                const int4 un = p.units[u];
                const int slot = STREAM ? 0 : i % a_slots;
                uint32_t a_base = 0;
                if constexpr (!STREAM) {   // the unit's resident R tile
                    const uint32_t use = (uint32_t)(i / a_slots);
                    if (!mbar_wait(a_full + slot, use & 1, abort_flag, p.wait_budget)) {
                        ok = false;
                        break;
                    }
                    if constexpr (CG2) {   // the peer's rows of the R tile
                        if (!mbar_wait_cluster(pa_full + slot, use & 1, abort_flag, p.wait_budget)) {
                            ok = false;
                            break;
                        }
                    }
                    tc_fence_after();
                    a_base = smem_u32(sA + slot * a_bytes);
                }
                for (int n = un.y; n < un.z && ok; n = tile_after<MASK>(p, un.x, n, un.z)) {
                    const uint32_t b = t % kAcc;
                    const bool freed = CG2 ? mbar_wait_cluster(acc_empty + b, ((t / kAcc) & 1) ^ 1, abort_flag,
                                                               p.wait_budget)
                                           : mbar_wait(acc_empty + b, ((t / kAcc) & 1) ^ 1, abort_flag, p.wait_budget);
                    if (!freed) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d_tmem = tmem_base + b * BN;
                    for (int c = 0; c < kc; ++c) {
                        if (!mbar_wait(full + stage, phase, abort_flag, p.wait_budget)) {
                            ok = false;
                            break;
                        }
                        if constexpr (CG2) {   // the peer's half of this stage
                            if (!mbar_wait_cluster(pfull + stage, phase, abort_flag, p.wait_budget)) {
                                ok = false;
                                break;
                            }
                        }
                        tc_fence_after();
                        const uint32_t a_addr =
                            STREAM ? smem_u32(sB + stage * kStageStride + kStageBytes) : a_base + c * 16384;
                        const uint32_t b_addr = smem_u32(sB + stage * kStageStride);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {   // 4 x 32 bytes of K per 128-byte chunk
                            const uint64_t ad = smem_desc_sw128(a_addr + k * 32), bd = smem_desc_sw128(b_addr + k * 32);
                            if constexpr (CG2 && FP8)
                                mma_f8_cg2(d_tmem, ad, bd, idesc, (c | k) != 0);
                            else if constexpr (CG2)
                                mma_f16_cg2(d_tmem, ad, bd, idesc, (c | k) != 0);
                            else if constexpr (FP8)
                                mma_f8(d_tmem, ad, bd, idesc, (c | k) != 0);
                            else
                                mma_f16(d_tmem, ad, bd, idesc, (c | k) != 0);
                        }
                        any_mma = true;
                        if constexpr (CG2)
                            mma_commit_cg2_mc(empty + stage, 3);   // both CTAs may refill their halves
                        else
                            mma_commit(empty + stage);
                        if (++stage == (uint32_t)stages) {
                            stage = 0;
                            phase ^= 1;
                        }
                    }
                    if (!ok) break;
                    if constexpr (CG2)
                        mma_commit_cg2_mc(acc_full + b, 3);   // both CTAs' rows are in their TMEM
                    else
                        mma_commit(acc_full + b);
                    ++t;
                }
                if (ok && !STREAM) {
                    if constexpr (CG2)
                        mma_commit_cg2_mc(a_empty + slot, 3);
                    else
                        mma_commit(a_empty + slot);
                }
            }
            if (!ok) raise_abort();
            // No MMA may still be running when TMEM is released. (A CTA that issued none -- one
            // that got no unit, or whose first wait ran out -- has nothing to wait for.)
            if (CG2 || any_mma) {
                if constexpr (CG2)
                    mma_commit_cg2(done);
                else
                    mma_commit(done);
                mbar_wait_plain(done, 0);
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int e = warp - 2;            // 0 .. kEpi-1
        const int quad = warp & 3;         // TMEM lanes this warp may access: 32*quad .. +31
        const int half = e >> 2;           // which HC-column part of the tile this warp owns
        const uint32_t lane_base = static_cast<uint32_t>(quad * 32) << 16;
        float *my_bt = s_beta + e * (kColSlots * HC);
        float *my_sx = s_sx + e * (kColSlots * kSubW);   // FP8 only
        float4 *my_cs = s_cst + e * (kColSlots * kSubW);
        uint2 *my_stg = s_stage + e * kStageCap;
        float *my_xch = s_xch + e * 32;
        uint32_t scnt = 0;
        constexpr int kPer = HC / 32;      // beta values a lane stages per tile (4 or 2)
        static_assert(kPer == 4 || kPer == 2, "an epilogue warp owns 128 or 64 columns");
        TileIter<MASK> cur, nxt;
        cur.start(p, ufirst, ustride, n_units);
        nxt = cur;
        nxt.next(p);

        auto stage_async = [&](const TileIter<MASK> &it, int s) {
            if (!it.valid) return;
            const int c0 = it.n * BN + half * HC;
            // the column data (beta [n_pad], chunk stats [n_pad / 32]) covers whole 256-column tiles
            if (!DL_CHECK(c0 + HC <= (p.nS + 255) / 256 * 256, 4, c0)) return;
            if constexpr (kPer == 4) {
                cp_async_16(my_bt + s * HC + lane * 4, p.beta + c0 + lane * 4);
                if (FP8 && lane == kSubW) cp_async_16(my_sx + s * kSubW, p.sc_s + (c0 >> 5));   // 4 chunk scales
            } else {
                cp_async_8(my_bt + s * HC + lane * 2, p.beta + c0 + lane * 2);
                if (FP8 && lane == kSubW) cp_async_8(my_sx + s * kSubW, p.sc_s + (c0 >> 5));    // 2 chunk scales
            }
            if (lane < kSubW) cp_async_16(my_cs + s * kSubW + lane, p.cstat + (c0 >> 5) + lane);
            cp_async_commit();
        };
        stage_async(cur, 0);
        cp_async_wait_all();
        __syncwarp();

        uint32_t t = 0;
        bool ok = true;
        float4 rp = make_float4(0.f, 0.f, 0.f, 0.f);
        float sq = 1.0f;          // FP8: this row's scale
        float theta = 0.f;        // top-k: this slot's threshold (k-th largest lower bound of h)
        float theta_row = 0.f;    // top-k: best threshold published by any slot of this row
        int tcnt = 0;             // top-k: this slot's list fill
        size_t sidx = 0;
        while (cur.valid) {
            const int r = (cur.un.x * kRowTiles + (int)crank) * 128 + quad * 32 + lane;
            if (cur.n == cur.un.y) {
                // per-row parameters cover whole R tiles (256-row tiles for SM pairs)
                if (DL_CHECK(r < (p.nR + kRowTiles * 128 - 1) / (kRowTiles * 128) * (kRowTiles * 128), 3, r))
                    rp = p.rowpar[r];
                if constexpr (FP8) sq = (r < p.nR) ? p.sc_r[r] : 1.0f;
                if constexpr (TOPK) {   // a unit owns its (row tile, split): start the slots fresh
                    sidx = (size_t)r * p.tk_slots + (size_t)cur.un.w * (kEpi / 4) + half;   // (split, column part)
                    theta = __int_as_float(0xff800000);
                    tcnt = 0;
                    if (r < p.nR) {
                        float *heap = p.tk_heap + sidx * (size_t)p.tk_k;
                        for (int i = 0; i < p.tk_k; ++i) heap[i] = __int_as_float(0xff800000);
                    }
                }
            }
            stage_async(nxt, (t & 1) ^ 1);   // the next tile's column data lands while this one is processed

            if constexpr (TOPK) {
                theta_row = __int_as_float(0xff800000);
                if (r < p.nR) theta_row = float_from_order_code(__ldcg(p.tk_row_theta + r));
            }
            const uint32_t b = t % kAcc;
            const int slot = t & 1;
            if (!mbar_wait(acc_full + b, (t / kAcc) & 1, abort_flag, p.wait_budget)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t tbase = tmem_base + lane_base + b * BN + half * HC;
            const float *beta = my_bt + slot * HC;
            const float *sxs = my_sx + slot * kSubW;
            const float4 *cst = my_cs + slot * kSubW;
            const int colw = cur.n * BN + half * HC;   // first column this warp owns in the tile

            // 64 columns [piece*64, piece*64+64) of this warp's half, values in v
            auto process64 = [&](uint32_t (&v)[64], int piece) {
                // FP8: h = fl(A s_q s_chunk - beta), one rounding (the scale product is an exact power of two)
                const float sc0 = FP8 ? sq * sxs[2 * piece] : 1.0f, sc1 = FP8 ? sq * sxs[2 * piece + 1] : 1.0f;
                const float4 cs0 = cst[2 * piece], cs1 = cst[2 * piece + 1];
                const float eh0 = __fmaf_ru(rp.z, cs0.x, __fmaf_ru(rp.w, cs0.y, cs0.z));
                const float eh1 = __fmaf_ru(rp.z, cs1.x, __fmaf_ru(rp.w, cs1.y, cs1.z));
                if (p.dump_h) {   // diagnostics: every pair's h and bound, at caller row order
#pragma unroll
                    for (int j = 0; j < 64; ++j) {
                        const int c = colw + piece * 64 + j;
                        if (r < p.nR && c < p.nS) {
                            const float h = __fmaf_rn(__uint_as_float(v[j]), j < 32 ? sc0 : sc1, -beta[piece * 64 + j]);
                            const size_t o = (size_t)p.orig_r[r] * p.nS + p.orig_s[c];
                            p.dump_h[o] = h;
                            p.dump_e[o] = j < 32 ? eh0 : eh1;
                        }
                    }
                }
                float tr0, tr1;
                if constexpr (TOPK) {   // candidate iff h + E (+ canonical slack rp.x) >= the best threshold
                    const float th = fmaxf(theta, theta_row);
                    tr0 = __fsub_rd(th, __fadd_ru(eh0, rp.x));
                    tr1 = __fsub_rd(th, __fadd_ru(eh1, rp.x));
                } else {
                    tr0 = __fsub_rd(rp.y, eh0);
                    tr1 = __fsub_rd(rp.y, eh1);
                }
                // Whole-chunk reject: with beta_j >= beta_min(chunk) and one scale s > 0 per chunk,
                // every h_j = fl(A_j s - beta_j) is <= fl_ru(max_j A_j * s - beta_min); rows are in
                // norm order, so beta_min is tight.
                const float mx0 = max_tree32(v, 0), mx1 = max_tree32(v, 32);
                const bool hit0 = __fmaf_ru(mx0, sc0, -cs0.w) >= tr0;
                const bool hit1 = __fmaf_ru(mx1, sc1, -cs1.w) >= tr1;
                if constexpr (TOPK) {
                    if (hit0 || hit1)
                        slow_topk(p, v, beta + piece * 64, __fadd_ru(eh0, rp.x), __fadd_ru(eh1, rp.x), hit0, hit1, r,
                                  colw + piece * 64, sidx, theta, tcnt, theta_row);
                } else {
                    if (__any_sync(0xffffffffu, hit0 || hit1)) {
                        const int c0 = colw + piece * 64;
                        scnt = slow_chunk<FP8>(p, v, 0, beta + piece * 64, sc0, __fadd_ru(rp.x, eh0),
                                               __fsub_rd(rp.y, eh0), hit0, r, c0, my_xch, my_stg, scnt);
                        scnt = slow_chunk<FP8>(p, v, 32, beta + piece * 64, sc1, __fadd_ru(rp.x, eh1),
                                               __fsub_rd(rp.y, eh1), hit1, r, c0 + 32, my_xch, my_stg, scnt);
                    }
                }
            };

            // One 32-column chunk ci of this warp's HC columns, values v[o .. o+31] (epsilon-join).
            auto eps_chunk = [&](auto &v, int o, int ci) {
                const float sc = FP8 ? sq * sxs[ci] : 1.0f;
                const float4 cs = cst[ci];
                const float eh = __fmaf_ru(rp.z, cs.x, __fmaf_ru(rp.w, cs.y, cs.z));
                if (p.dump_h) {   // diagnostics: every pair's h and bound, at caller row order
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int c = colw + ci * 32 + j;
                        if (r < p.nR && c < p.nS) {
                            const float h = __fmaf_rn(__uint_as_float(v[o + j]), sc, -beta[ci * 32 + j]);
                            const size_t oi = (size_t)p.orig_r[r] * p.nS + p.orig_s[c];
                            p.dump_h[oi] = h;
                            p.dump_e[oi] = eh;
                        }
                    }
                }
                // whole-chunk reject (see process64)
                const float mx = max_tree32(v, o);
                const bool hit = __fmaf_ru(mx, sc, -cs.w) >= __fsub_rd(rp.y, eh);
                if (__any_sync(0xffffffffu, hit))
                    scnt = slow_chunk<FP8>(p, v, o, beta + ci * 32, sc, __fadd_ru(rp.x, eh), __fsub_rd(rp.y, eh), hit,
                                           r, colw + ci * 32, my_xch, my_stg, scnt);
            };
            auto release_acc = [&]() {
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {   // TMEM buffer free; the rest is in registers
                    if constexpr (CG2) {
                        if (leader)
                            mbar_arrive(acc_empty + b);
                        else
                            mbar_arrive_remote(mapa_shared(acc_empty + b, 0u));
                    } else {
                        mbar_arrive(acc_empty + b);
                    }
                }
            };
            // Top-k, one 32-column chunk ci (BF16 only: scale 1): the columns whose upper bound
            // reaches the best threshold go to the slot's list, their lower bounds to its heap.
            auto topk_chunk = [&](auto &v, int o, int ci) {
                const float4 cs = cst[ci];
                const float ehs = __fadd_ru(__fmaf_ru(rp.z, cs.x, __fmaf_ru(rp.w, cs.y, cs.z)), rp.x);
                const float mx = max_tree32(v, o);
                if (__fsub_ru(mx, cs.w) >= __fsub_rd(fmaxf(theta, theta_row), ehs) && r < p.nR) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int c = colw + ci * 32 + j;
                        const float h = __uint_as_float(v[o + j]) - beta[ci * 32 + j];
                        const float U = __fadd_ru(h, ehs);
                        if (c < p.nS && U >= fmaxf(theta, theta_row)) {
                            const float2 stt = topk_insert(p, sidx, r, c, U, __fsub_rd(h, ehs), theta, tcnt, theta_row);
                            theta = stt.x;
                            tcnt = __float_as_int(stt.y);
                        }
                    }
                }
            };
            if constexpr (kEpi == 16) {
                // 64 columns per warp, 32 at a time: the three other epilogue warps of this SM
                // sub-partition hide each load's latency
                uint32_t vq[32];
                tmem_ld_32x32b_x32(tbase, vq);
                tmem_ld_wait_regs(vq);
                if constexpr (TOPK)
                    topk_chunk(vq, 0, 0);
                else
                    eps_chunk(vq, 0, 0);
                tmem_ld_32x32b_x32(tbase + 32, vq);
                tmem_ld_wait_regs(vq);
                release_acc();
                if constexpr (TOPK)
                    topk_chunk(vq, 0, 1);
                else
                    eps_chunk(vq, 0, 1);
            } else {
            // One 64-column load at a time: the other epilogue warp on this SM
            // sub-partition hides the TMEM load latency.
            uint32_t va[64];
            if constexpr (HC == 128) {
                tmem_ld_32x32b_x64(tbase, va);
                tmem_ld_wait_regs(va);
                process64(va, 0);
                tmem_ld_32x32b_x64(tbase + 64, va);
                tmem_ld_wait_regs(va);
            } else {
                tmem_ld_32x32b_x64(tbase, va);
                tmem_ld_wait_regs(va);
            }
            release_acc();
            process64(va, HC == 128 ? 1 : 0);
            }
            if constexpr (TOPK) {
                if (cur.n + 1 == cur.un.z && r < p.nR) {   // last tile of the unit: publish the slot
                    p.tk_theta[sidx] = theta;
                    p.tk_cnt[sidx] = tcnt;
                }
            }
            // the next tile's column data is in the other slot
            cp_async_wait_all();
            __syncwarp();
            cur = nxt;
            nxt.next(p);
            ++t;
        }
        cp_async_wait_all();   // no staged column data may still be in flight when the CTA ends
        if constexpr (!TOPK) flush_stage(p, my_stg, scnt);
        if (!ok) raise_abort();
    }

    __syncthreads();
    // CG2: neither CTA of the pair releases its TMEM or exits while the other may still use
    // it -- the leader's MMAs write the peer's TMEM and read its shared memory, and the peer
    // arrives on the leader's barriers. Every path of every thread reaches this point.
    if constexpr (CG2) cluster_sync_all();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc<CG2>(tmem_base, kTmemCols);
    }
}

static size_t tc_extra_bytes(int BN, bool fp8, bool wide)
{
    // per epilogue warp (owning HC columns): kColSlots x HC floats of beta, kColSlots x HC/32 chunk
    // stats, the candidate buffer and (FP8) kColSlots x HC/32 chunk scales; then 48 barrier / flag
    // words and 32 exchange floats per epilogue warp
    const size_t epi = (size_t)tc_epi_warps(wide), hc = (size_t)BN * 4 / epi;
    return epi * (kColSlots * hc * 4 + kColSlots * (hc / 32) * 16 + kStageCap * 8 + (fp8 ? kColSlots * (hc / 32) * 4 : 0)) +
           48 * 8 + epi * 32 * 4;
}

// One S stage per CTA: a 128-byte K chunk of the CTA's rows of an S tile (all BN rows, or
// BN/2 for a CTA pair).
static size_t tc_stage_bytes(int BN, bool cg2) { return (size_t)(cg2 ? BN / 2 : BN) * 128; }

// a_slots == 0: streamed R chunks, 16 KB more per stage and no resident tile
static size_t tc_smem_bytes(int BN, int kc, int stages, int a_slots, bool fp8, bool cg2, bool wide)
{
    return 1024 + (size_t)a_slots * kc * 16384 + (size_t)stages * (tc_stage_bytes(BN, cg2) + (a_slots ? 0 : 16384)) +
           tc_extra_bytes(BN, fp8, wide);
}

// Shared-memory plan: two A slots when that still leaves at least three S stages, else one;
// with `stream` (the one-SM epsilon-join), a plan that would be left with fewer than three
// stages beside one resident R tile streams the R tile's chunks with the S chunks instead
// (a_slots = 0).
void tc_plan(int BN, int kc, int *stages, int *a_slots, bool fp8, bool cg2, bool wide, bool stream)
{
    const long cap = 232448;
    for (int slots = 2; slots >= 1; --slots) {
        const long avail = cap - 1024 - (long)tc_extra_bytes(BN, fp8, wide) - (long)slots * kc * 16384;
        long s = avail / (long)tc_stage_bytes(BN, cg2);
        if (s > 8) s = 8;
        if (s >= 3 || slots == 1) {
            *stages = (int)s;
            *a_slots = slots;
            if (s >= 3 || !stream || cg2) return;
            break;
        }
    }
    long s = (cap - 1024 - (long)tc_extra_bytes(BN, fp8, wide)) / (long)(tc_stage_bytes(BN, cg2) + 16384);
    if (s > 8) s = 8;
    *stages = (int)s;
    *a_slots = 0;
}

static std::atomic<long long> g_wait_budget{0};

long long tc_wait_budget()
{
    const long long b = g_wait_budget.load(std::memory_order_relaxed);
    return b > 0 ? b : kWaitBudgetClocks;
}

template <int BN, bool TOPK, bool FP8, bool CG2, bool WIDE = false, bool MASK = false, bool STREAM = false>
static int launch_one(const TcLaunch &L, size_t smem, cudaStream_t st, int *grid_out)
{
    auto kern = tc_join_kernel<BN, TOPK, FP8, CG2, WIDE, MASK, STREAM>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(tc_join_kernel)");
    TcParams p = L.p;
    p.wait_budget = tc_wait_budget();
    if constexpr (CG2) {
        cudaLaunchConfig_t cfg = {};
        cfg.blockDim = dim3(tc_threads(WIDE));
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        // persistent pairs: no more than can be resident at once (GPCs may leave an SM unpaired)
        cfg.gridDim = dim3(2);
        int pairs = 0;
        e = cudaOccupancyMaxActiveClusters(&pairs, kern, &cfg);
        if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveClusters(tc_join_kernel)");
        if (pairs < 1) {
            set_error("tensor-core join: no CTA pair fits on this device");
            return DL_EUNSUPPORTED;
        }
        const int want = std::max(1, L.grid / 2);
        cfg.gridDim = dim3((unsigned)(2 * std::min(want, pairs)));
        e = cudaLaunchKernelEx(&cfg, kern, *L.tmA, *L.tmB, p);
        if (e != cudaSuccess) return cuda_fail(e, "tc_join_kernel (CTA pairs) launch");
        if (grid_out) *grid_out = (int)cfg.gridDim.x;
    } else {
        kern<<<L.grid, tc_threads(WIDE), smem, st>>>(*L.tmA, *L.tmB, p);
        if (grid_out) *grid_out = L.grid;
    }
    return DL_OK;
}

int launch_tc_join(const TcLaunch &L, cudaStream_t st, bool topk, bool fp8, int *grid_out)
{
    if (topk && fp8) {
        set_error("top-k runs on the BF16 path only");
        return DL_EUNSUPPORTED;
    }
    if ((L.cg2 && (topk || L.BN != 256 || L.wide)) || (L.wide && L.BN != 256)) {
        set_error("tensor-core join: CTA pairs serve the 256-column epsilon-join, the wide epilogue 256-column tiles");
        return DL_EUNSUPPORTED;
    }
    const size_t smem = tc_smem_bytes(L.BN, L.p.kc, L.p.stages, L.p.a_slots, fp8, L.cg2, L.wide);
    if (L.p.stages < 2 || smem > 232448) {
        set_error("tensor-core join: no shared-memory plan for d=%d, tile %d", L.p.kc * 64, L.BN);
        return DL_EUNSUPPORTED;
    }
    int rc;
    if (L.p.a_slots == 0) {   // streamed R chunks (tc_plan with stream): the one-SM epsilon-join
        if (topk || L.cg2 || L.p.tile_mask) {
            set_error("tensor-core join: streamed R chunks serve the dense one-SM epsilon-join");
            return DL_EUNSUPPORTED;
        }
        if (L.wide)
            rc = fp8 ? launch_one<256, false, true, false, true, false, true>(L, smem, st, grid_out)
                     : launch_one<256, false, false, false, true, false, true>(L, smem, st, grid_out);
        else if (L.BN == 256)
            rc = fp8 ? launch_one<256, false, true, false, false, false, true>(L, smem, st, grid_out)
                     : launch_one<256, false, false, false, false, false, true>(L, smem, st, grid_out);
        else if (L.BN == 128)
            rc = fp8 ? launch_one<128, false, true, false, false, false, true>(L, smem, st, grid_out)
                     : launch_one<128, false, false, false, false, false, true>(L, smem, st, grid_out);
        else {
            set_error("tensor-core tile width %d not supported (128 or 256)", L.BN);
            return DL_EINVAL;
        }
    } else if (L.p.tile_mask) {   // the pruned join: units and their count built on the device
        if (topk || L.cg2 || !L.p.n_units_dev) {
            set_error("tensor-core join: a tile mask serves the one-SM epsilon-join with device-built units");
            return DL_EUNSUPPORTED;
        }
        if (L.wide)
            rc = fp8 ? launch_one<256, false, true, false, true, true>(L, smem, st, grid_out)
                     : launch_one<256, false, false, false, true, true>(L, smem, st, grid_out);
        else if (L.BN == 256)
            rc = fp8 ? launch_one<256, false, true, false, false, true>(L, smem, st, grid_out)
                     : launch_one<256, false, false, false, false, true>(L, smem, st, grid_out);
        else if (L.BN == 128)
            rc = fp8 ? launch_one<128, false, true, false, false, true>(L, smem, st, grid_out)
                     : launch_one<128, false, false, false, false, true>(L, smem, st, grid_out);
        else {
            set_error("tensor-core tile width %d not supported (128 or 256)", L.BN);
            return DL_EINVAL;
        }
    } else if (L.cg2)
        rc = fp8 ? launch_one<256, false, true, true>(L, smem, st, grid_out) : launch_one<256, false, false, true>(L, smem, st, grid_out);
    else if (L.wide)
        rc = topk ? launch_one<256, true, false, false, true>(L, smem, st, grid_out)
                  : (fp8 ? launch_one<256, false, true, false, true>(L, smem, st, grid_out)
                         : launch_one<256, false, false, false, true>(L, smem, st, grid_out));
    else if (L.BN == 256)
        rc = topk ? launch_one<256, true, false, false>(L, smem, st, grid_out)
                  : (fp8 ? launch_one<256, false, true, false>(L, smem, st, grid_out)
                         : launch_one<256, false, false, false>(L, smem, st, grid_out));
    else if (L.BN == 128)
        rc = topk ? launch_one<128, true, false, false>(L, smem, st, grid_out)
                  : (fp8 ? launch_one<128, false, true, false>(L, smem, st, grid_out)
                         : launch_one<128, false, false, false>(L, smem, st, grid_out));
    else {
        set_error("tensor-core tile width %d not supported (128 or 256)", L.BN);
        return DL_EINVAL;
    }
    if (rc) return rc;
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tc_join_kernel launch");
    return DL_OK;
}

}  // namespace dl

// Diagnostics: shorten the abortable pipeline waits of every tensor-core kernel
// launched from now on (0 restores the default), so tests can make a healthy
// join's wait run out and exercise the abort path.
extern "C" int dl_debug_set_wait_budget(int64_t clocks)
{
    dl::clear_error();
    if (clocks < 0) {
        dl::set_error("dl_debug_set_wait_budget: clocks must be >= 0 (got %lld)", (long long)clocks);
        return DL_EINVAL;
    }
    dl::g_wait_budget.store(clocks, std::memory_order_relaxed);
    return DL_OK;
}

DL_CHECK_READER(join_tc)
