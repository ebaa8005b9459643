// prune.cu -- the exact pruned similarity join (the GPU counterpart of the paper's
// on-the-fly Ball-Tree join, Sec. 5 and Sec. 7.3) and the clustered store order it needs.
//
// Pruning: every R tile (128 store rows) and S tile (BN rows) gets bounding balls, one per
// run of equal cluster labels in the tile (or one for the whole tile): a centre c (the
// FP32-rounded mean of the run's rows) and a radius r >= max ||x - c|| (FP64, rounded up).
// For q in one ball and x in another the triangle inequality gives ||q - x|| >= ||c_1 -
// c_2|| - r_1 - r_2, so a tile pair all of whose ball pairs have a lower bound, shrunk by
// safety margins for its own FP32 evaluation, above eps cannot hold a pair: its canonical
// D exceeds eps^2 as well. Only the surviving tile pairs become work units of
// the unchanged tensor-core join, so the result is the exact set and the skipped tiles
// cost no MMA, no S traffic and no epilogue.
//
// Clustering (dl_store_cluster): balls are tight only when a tile holds one compact
// group of rows, so the store is re-ordered by a few k-means iterations whose
// assignment step is the library's own exact top-1 join against the centroids.
#include <algorithm>
#include <vector>

#include "kernels.h"

namespace dl {

namespace {

constexpr int kBallThreads = 128;

constexpr int kMaxSeg = 4;   // bounding balls per tile

// One CTA per tile of `rows` store rows. With cluster labels, the tile's rows are cut into
// its runs of equal label (at most kMaxSeg; a tile with more runs keeps one ball), and each
// run gets a ball: the FP32-rounded mean as centre and an FP64 radius bound rounded up to
// FP32. Without labels the whole tile is one run. Centres are written transposed,
// centre[(u * d + k) * nt + tile], so that neighbouring tiles are neighbouring words.
__global__ void __launch_bounds__(kBallThreads)
    k_tile_balls(const float *__restrict__ x, const int32_t *__restrict__ label, int64_t n, int d, int rows, int nt,
                 float *__restrict__ centre, float *__restrict__ radius, int *__restrict__ nseg)
{
    extern __shared__ float sc[];   // [d] the current centre
    __shared__ double red[kBallThreads / 32];
    __shared__ int seg_lo[kMaxSeg + 1];
    __shared__ int s_nseg;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * rows;
    const int64_t r1 = (r0 + rows < n) ? r0 + rows : n;
    if (threadIdx.x == 0) {
        int k = 1;
        seg_lo[0] = 0;
        if (label) {
            for (int64_t r = r0 + 1; r < r1 && k <= kMaxSeg; ++r)
                if (label[r] != label[r - 1]) {
                    if (k < kMaxSeg) seg_lo[k] = (int)(r - r0);
                    ++k;
                }
            if (k > kMaxSeg) k = 1;   // too many runs: one ball for the tile
        }
        seg_lo[k] = (int)(r1 - r0);
        s_nseg = k;
        nseg[blockIdx.x] = k;
    }
    __syncthreads();
    const int ns = s_nseg;
    for (int sgi = 0; sgi < ns; ++sgi) {
        const int64_t a = r0 + seg_lo[sgi], b = r0 + seg_lo[sgi + 1];
        for (int k = threadIdx.x; k < d; k += kBallThreads) {
            double s = 0.0;
            for (int64_t r = a; r < b; ++r) s += (double)x[r * d + k];
            const float c = (float)(s / (double)(b - a));
            sc[k] = c;
            centre[((int64_t)sgi * d + k) * nt + blockIdx.x] = c;
        }
        __syncthreads();
        // one warp per row, lanes over the columns
        double mx = 0.0;
        for (int64_t r = a + wid; r < b; r += kBallThreads / 32) {
            double s = 0.0;
            for (int k = lane; k < d; k += 32) {
                const double t = (double)x[r * d + k] - (double)sc[k];
                s += t * t;
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            mx = fmax(mx, s);
        }
        if (lane == 0) red[wid] = mx;
        __syncthreads();
        if (threadIdx.x == 0) {
            double m = red[0];
            for (int w = 1; w < kBallThreads / 32; ++w) m = fmax(m, red[w]);
            // sqrt of the FP64 maximum, widened for the rounding of the FP64 sums (relative
            // error far below 1e-12) and rounded up to FP32
            radius[(int64_t)blockIdx.x * kMaxSeg + sgi] = __double2float_ru(sqrt(m) * (1.0 + 1e-9) + 1e-30);
        }
        __syncthreads();
    }
}

// Word m * ntw + t / 32, bit t % 32 of the mask is 1 unless every ball of R tile m lies
// provably farther than eps from every ball of S tile t. One CTA row per R tile (its balls
// staged in shared memory), one thread per S tile. Centre distances are FP32 sums
// (relative error below (d + 2) 2^-24 < 1e-4 / 2 for d <= 1024), so they are shrunk by 1e-4
// before the radii are subtracted.
__global__ void __launch_bounds__(256)
    k_prune_mask(const float *__restrict__ cR, const float *__restrict__ rR, const int *__restrict__ nR_seg, int mt,
                 const float *__restrict__ cS, const float *__restrict__ rS, const int *__restrict__ nS_seg, int nt,
                 int d, float e2_up, uint32_t *__restrict__ mask)
{
    extern __shared__ float cm[];   // [kMaxSeg][d] the balls of R tile m
    const int m = blockIdx.y;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int na = nR_seg[m];
    for (int i = threadIdx.x; i < na * d; i += blockDim.x) cm[i] = cR[(int64_t)i * mt + m];
    __syncthreads();
    bool keep = false;
    if (t < nt) {
        const int nb = nS_seg[t];
        for (int v = 0; v < nb && !keep; ++v) {
            // one pass over S ball v's centre serves every ball of the R tile
            float su[kMaxSeg] = {0.f, 0.f, 0.f, 0.f};
            const float *b = cS + (int64_t)v * d * nt + t;
#pragma unroll 8
            for (int k = 0; k < d; ++k) {
                const float bv = __ldg(b + (int64_t)k * nt);
#pragma unroll
                for (int u = 0; u < kMaxSeg; ++u)
                    if (u < na) {
                        const float w = cm[u * d + k] - bv;
                        su[u] = fmaf(w, w, su[u]);
                    }
            }
#pragma unroll
            for (int u = 0; u < kMaxSeg; ++u)
                if (u < na) {
                    const float lower = sqrtf(su[u]) * (1.0f - 1e-4f) - rR[m * kMaxSeg + u] - rS[t * kMaxSeg + v];
                    keep |= !(lower > 0.f && lower * lower > e2_up);
                }
        }
    }
    const unsigned word = __ballot_sync(0xffffffffu, keep);
    const int ntw = (nt + 31) >> 5;
    if ((threadIdx.x & 31) == 0 && t < nt) mask[(int64_t)m * ntw + (t >> 5)] = word;
}

// First S tile of R tile m a self-join (upper) computes: tiles wholly at or below the diagonal
// hold no pair c > r.
__host__ __device__ __forceinline__ int first_upper_tile(int m, int BN, bool upper)
{
    if (!upper) return 0;
    const long long num = (long long)m * 128 + 2 - BN;
    return num <= 0 ? 0 : (int)((num + BN - 1) / BN);
}

// Units of the pruned join from the tile mask, in one CTA: block pair i = b * mt + m (S-range-
// major, as the dense units) covers S tiles [64 b, 64 b + 64) of R tile m from its first upper
// tile on. A pair with a surviving tile becomes unit {m, first kept, last kept + 1, 0}; a CTA-
// wide exclusive scan of the keep flags places the units in order. Also counts the surviving
// tiles. Grid: one CTA of 1024 threads.
__global__ void __launch_bounds__(1024)
    k_prune_units(const uint32_t *__restrict__ mask, int mt, int nt, int ntw, int BN, int upper, int4 *__restrict__ units,
                  int *__restrict__ n_units, unsigned long long *__restrict__ kept)
{
    __shared__ int s_warp[32];
    __shared__ int s_base;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const long long npairs = (long long)((nt + 63) / 64) * mt;
    if (tid == 0) s_base = 0;
    unsigned long long my_kept = 0;
    __syncthreads();
    for (long long c0 = 0; c0 < npairs; c0 += 1024) {
        const long long i = c0 + tid;
        int m = 0, first = -1, last = -1;
        if (i < npairs) {
            const int b = (int)(i / mt);
            m = (int)(i % mt);
            const int lo = max(b * 64, first_upper_tile(m, BN, upper != 0)), hi = min(b * 64 + 64, nt);
            for (int wd = lo >> 5; lo < hi && wd <= (hi - 1) >> 5; ++wd) {
                uint32_t word = mask[(size_t)m * ntw + wd];
                const int w0 = wd * 32;
                if (lo > w0) word &= ~0u << (lo - w0);
                if (hi < w0 + 32) word &= ~0u >> (32 - (hi - w0));
                if (word) {
                    if (first < 0) first = w0 + __ffs((int)word) - 1;
                    last = w0 + 31 - __clz((int)word);
                    my_kept += (unsigned long long)__popc(word);
                }
            }
        }
        const bool keep = first >= 0;
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) s_warp[w] = __popc(bal);
        __syncthreads();
        if (w == 0) {   // exclusive scan of the 32 warp counts
            const int v = s_warp[lane];
            int x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            s_warp[lane] = x - v;
        }
        __syncthreads();
        if (keep) units[s_base + s_warp[w] + __popc(bal & ((1u << lane) - 1u))] = make_int4(m, first, last + 1, 0);
        __syncthreads();
        if (tid == 1023) s_base += s_warp[31] + __popc(bal);
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_kept += __shfl_xor_sync(0xffffffffu, my_kept, o);
    if (lane == 0 && my_kept) atomicAdd(kept, my_kept);
    if (tid == 0) *n_units = s_base;
}

__global__ void __launch_bounds__(256)
    k_label_of_rows(const int64_t *__restrict__ best, const int32_t *__restrict__ orig, int64_t n, int32_t *label)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        label[i] = (int32_t)best[orig[i]];
}

__global__ void __launch_bounds__(256)
    k_centroid_accum(const float *__restrict__ x, const int32_t *__restrict__ label, int64_t n, int d, float *sums,
                     unsigned *counts)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w; r < n; r += nw) {
        const int c = label[r];
        for (int k = lane; k < d; k += 32) atomicAdd(sums + (int64_t)c * d + k, x[r * d + k]);
        if (lane == 0) atomicAdd(counts + c, 1u);
    }
}

__global__ void __launch_bounds__(256)
    k_centroid_update(float *centres, const float *__restrict__ sums, const unsigned *__restrict__ counts, int K, int d)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)K * d) return;
    const unsigned c = counts[i / d];
    if (c) centres[i] = sums[i] / (float)c;   // an empty cluster keeps its centre
}

__global__ void __launch_bounds__(256)
    k_gather_centres(const float *__restrict__ x, int64_t n, int d, int K, float *centres, int64_t *ids)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)K * d) return;
    const int c = (int)(i / d), k = (int)(i - (int64_t)c * d);
    // rows spread pseudo-randomly over the store (the store is in norm order, so evenly spaced
    // rows would seed by norm): c * 1000003 mod n, distinct for distinct c when n is not a
    // multiple of that prime, and deterministic
    const int64_t row = (int64_t)(((unsigned long long)c * 1000003ull) % (unsigned long long)n);
    centres[i] = x[row * d + k];
    if (k == 0) ids[c] = c;
}

__global__ void __launch_bounds__(256) k_count_labels(const int32_t *__restrict__ label, int64_t n, unsigned *hist)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(hist + label[i], 1u);
}

// Exclusive prefix sum of hist[0..K) in place (one CTA).
__global__ void __launch_bounds__(1024) k_scan_labels(unsigned *hist, int K)
{
    __shared__ unsigned warp_tot[32];
    __shared__ unsigned carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int b0 = 0; b0 < K; b0 += 1024) {
        const int b = b0 + threadIdx.x;
        const unsigned x = b < K ? hist[b] : 0u;
        unsigned v = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) warp_tot[wid] = v;
        __syncthreads();
        if (wid == 0) {
            unsigned t = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned u = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += u;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        const unsigned incl = v + (wid ? warp_tot[wid - 1] : 0u) + carry;
        if (b < K) hist[b] = incl - x;
        __syncthreads();
        if (threadIdx.x == 1023) carry = incl;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256)
    k_scatter_labels(const int32_t *__restrict__ label, int64_t n, unsigned *cursor, int32_t *perm)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        perm[atomicAdd(cursor + label[i], 1u)] = (int32_t)i;
}

__global__ void __launch_bounds__(256)
    k_compose_orig(const int32_t *__restrict__ in_orig, const int32_t *__restrict__ perm, int64_t n, int32_t *out_orig)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out_orig[i] = in_orig[perm[i]];
}

__global__ void __launch_bounds__(256)
    k_permute_labels(const int32_t *__restrict__ lab, const int32_t *__restrict__ perm, int64_t n, int32_t *out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = lab[perm[i]];
}

int grid_of(int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)device_sm_count() * 8));
}

// The balls of a store's tiles of `rows` rows: computed once per store and tile height, then
// kept with the store (stores are immutable).
int tile_balls(Store *s, int rows, cudaStream_t st, const Store::BallCache **out)
{
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto &b : s->balls)
            if (b.rows == rows) {
                *out = &b;
                return DL_OK;
            }
    }
    const int64_t nt = (s->n + rows - 1) / rows;
    const int d = s->d;
    const size_t bc = ((size_t)nt * kMaxSeg * d * 4 + 255) & ~size_t(255), br = ((size_t)nt * kMaxSeg * 4 + 255) & ~size_t(255),
                 bn = ((size_t)nt * 4 + 255) & ~size_t(255);
    void *blk = nullptr;
    int rc = dev_alloc(&blk, bc + br + bn, st);
    if (rc) return rc;
    float *centre = (float *)blk, *radius = (float *)((char *)blk + bc);
    int *nseg = (int *)((char *)blk + bc + br);
    k_tile_balls<<<(unsigned)nt, kBallThreads, (size_t)d * sizeof(float), st>>>(s->x32, s->clabel, s->n, d, rows,
                                                                                (int)nt, centre, radius, nseg);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // published only once complete
    if (e != cudaSuccess) {
        dev_free(blk, st);
        return cuda_fail(e, "k_tile_balls");
    }
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto &b : s->balls)
        if (b.rows == rows) {   // another thread got there first
            dev_free(blk, st);
            *out = &b;
            return DL_OK;
        }
    Store::BallCache *slot = &s->balls[0];
    if (s->balls[0].rows) slot = &s->balls[1];
    if (slot->blk) dev_free(slot->blk, st);   // both slots taken: replace the second
    slot->rows = rows;
    slot->blk = blk;
    slot->centre = centre;
    slot->radius = radius;
    slot->nseg = nseg;
    *out = slot;
    return DL_OK;
}

}  // namespace

// Work units of the tile pairs that survive the ball test, built on the device (the tile mask,
// then k_prune_units); nothing is read back, so the join launches right after.
int prune_units(const dl_store *R, const dl_store *S, bool upper, int BN, double e2, cudaStream_t st, PruneUnits *pu)
{
    *pu = PruneUnits();
    const int mt = (int)((R->n + 127) / 128), nt = (int)((S->n + BN - 1) / BN);
    if (mt == 0 || nt == 0) return DL_OK;
    for (int m = 0; m < mt; ++m) pu->total += std::max(0, nt - first_upper_tile(m, BN, upper));
    const int d = R->d;
    const int ntw = (nt + 31) / 32;
    const size_t n_words = (size_t)mt * ntw;
    const int64_t cap = (int64_t)((nt + 63) / 64) * mt;
    const Store::BallCache *bR = nullptr, *bS = nullptr;
    int rc = tile_balls(const_cast<dl_store *>(R), 128, st, &bR);
    if (!rc) rc = tile_balls(const_cast<dl_store *>(S), BN, st, &bS);
    if (rc) return rc;
    const size_t b_units = ((size_t)cap * sizeof(int4) + 255) & ~(size_t)255;
    const size_t b_mask = (n_words * 4 + 255) & ~(size_t)255;
    void *blk = nullptr;
    rc = dev_alloc(&blk, b_units + b_mask + 256, st);
    if (rc) return rc;
    int4 *units = (int4 *)blk;
    uint32_t *mask = (uint32_t *)((char *)blk + b_units);
    int *count = (int *)((char *)blk + b_units + b_mask);
    unsigned long long *kept = (unsigned long long *)(count + 2);
    cudaError_t e = cudaMemsetAsync(count, 0, 16, st);
    if (e == cudaSuccess) {
        const float e2_up = std::isinf(e2) ? __builtin_inff() : f32_ru(e2 * (1.0 + 1e-6) + 1e-37);
        const dim3 grid((unsigned)((nt + 255) / 256), (unsigned)mt);
        k_prune_mask<<<grid, 256, (size_t)kMaxSeg * d * sizeof(float), st>>>(bR->centre, bR->radius, bR->nseg, mt,
                                                                              bS->centre, bS->radius, bS->nseg, nt, d,
                                                                              e2_up, mask);
        k_prune_units<<<1, 1024, 0, st>>>(mask, mt, nt, ntw, BN, upper ? 1 : 0, units, count, kept);
        count_launch(2);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        dev_free(blk, st);
        return cuda_fail(e, "prune units");
    }
    pu->block = blk;
    pu->units = units;
    pu->cap = (int)cap;
    pu->count = count;
    pu->mask = mask;
    pu->ntw = ntw;
    pu->kept = kept;
    return DL_OK;
}

}  // namespace dl

using namespace dl;

extern "C" int dl_store_cluster(const dl_store *in, int32_t n_clusters, int32_t iters, dl_store **out,
                                void *cuda_stream)
{
    dl::NvtxScope nvtx_scope("dl_store_cluster");
    clear_error();
    if (!in || !out) {
        set_error("dl_store_cluster: NULL argument");
        return DL_EINVAL;
    }
    *out = nullptr;
    if (n_clusters < 1 || iters < 0 || iters > 100) {
        set_error("dl_store_cluster: n_clusters must be >= 1 and iters in [0, 100]");
        return DL_EINVAL;
    }
    int dev = -1;
    DL_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != in->device) {
        set_error("dl_store_cluster: store lives on device %d but device %d is current", in->device, dev);
        return DL_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int64_t n = in->n;
    const int d = in->d;
    const int K = (int)std::min<int64_t>(n_clusters, std::max<int64_t>(n, 1));
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t b_c = al((size_t)K * d * 4), b_cid = al((size_t)K * 8), b_sum = al((size_t)K * d * 4),
                 b_cnt = al((size_t)K * 4), b_best = al((size_t)std::max<int64_t>(n, 1) * 8),
                 b_d2 = al((size_t)std::max<int64_t>(n, 1) * 8), b_lab = al((size_t)std::max<int64_t>(n, 1) * 4),
                 b_perm = al((size_t)std::max<int64_t>(n, 1) * 4);
    void *blk = nullptr;
    int rc = dev_alloc(&blk, b_c + b_cid + b_sum + b_cnt + b_best + b_d2 + b_lab + b_perm, st);
    if (rc) return rc;
    char *p = (char *)blk;
    float *cent = (float *)p;
    int64_t *cid = (int64_t *)(p + b_c);
    float *sums = (float *)(p + b_c + b_cid);
    unsigned *cnt = (unsigned *)(p + b_c + b_cid + b_sum);
    int64_t *best = (int64_t *)(p + b_c + b_cid + b_sum + b_cnt);
    double *bd2 = (double *)(p + b_c + b_cid + b_sum + b_cnt + b_best);
    int32_t *lab = (int32_t *)(p + b_c + b_cid + b_sum + b_cnt + b_best + b_d2);
    int32_t *perm = (int32_t *)(p + b_c + b_cid + b_sum + b_cnt + b_best + b_d2 + b_lab);
    cudaError_t e = cudaSuccess;
    if (n > 0) {
        k_gather_centres<<<(unsigned)(((int64_t)K * d + 255) / 256), 256, 0, st>>>(in->x32, n, d, K, cent, cid);
        count_launch();
        e = cudaGetLastError();
    }
    dl_join_opts o;
    dl_join_opts_default(&o);
    o.cuda_stream = cuda_stream;
    o.precision = DL_PREC_AUTO;
    for (int it = 0; n > 0 && e == cudaSuccess && !rc && it <= iters; ++it) {
        // assignment: the exact top-1 join of every row against the current centres
        dl_store *C = nullptr;
        rc = store_create_impl(&C, cid, cent, K, d, DL_MEM_DEVICE, cuda_stream, nullptr);
        if (rc) break;
        rc = topk_core(in, C, 1, nullptr, nullptr, best, bd2, o, st, nullptr);
        cudaStreamSynchronize(st);
        dl_store_destroy(C);
        if (rc) break;
        k_label_of_rows<<<grid_of(n), 256, 0, st>>>(best, in->orig, n, lab);
        count_launch();
        if (it == iters) break;
        // update: the mean of each cluster's rows
        e = cudaMemsetAsync(sums, 0, b_sum + b_cnt, st);
        if (e != cudaSuccess) break;
        k_centroid_accum<<<grid_of(n * 32), 256, 0, st>>>(in->x32, lab, n, d, sums, cnt);
        k_centroid_update<<<(unsigned)(((int64_t)K * d + 255) / 256), 256, 0, st>>>(cent, sums, cnt, K, d);
        count_launch(2);
        e = cudaGetLastError();
    }
    if (!rc && e == cudaSuccess && n > 0) {
        // store order: rows grouped by cluster (counting sort of the labels)
        e = cudaMemsetAsync(cnt, 0, b_cnt, st);
        if (e == cudaSuccess) {
            k_count_labels<<<grid_of(n), 256, 0, st>>>(lab, n, cnt);
            k_scan_labels<<<1, 1024, 0, st>>>(cnt, K);
            k_scatter_labels<<<grid_of(n), 256, 0, st>>>(lab, n, cnt, perm);
            count_launch(3);
            e = cudaGetLastError();
        }
    }
    if (!rc && e != cudaSuccess) rc = cuda_fail(e, "dl_store_cluster");
    dl_store *s = nullptr;
    if (!rc) {
        rc = store_create_impl(&s, in->ids, in->x32, n, d, DL_MEM_DEVICE, cuda_stream, n > 0 ? perm : nullptr);
    }
    int32_t *clabel = nullptr;
    if (!rc && n > 0) rc = dev_alloc((void **)&clabel, (size_t)n * 4, st);
    if (!rc && n > 0) {
        // caller rows follow the input store's caller rows; each row keeps its cluster label
        k_compose_orig<<<grid_of(n), 256, 0, st>>>(in->orig, perm, n, s->orig);
        k_permute_labels<<<grid_of(n), 256, 0, st>>>(lab, perm, n, clabel);
        count_launch();
        count_launch();
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "dl_store_cluster orig");
    }
    dev_free(blk, st);
    if (rc) {
        if (clabel) dev_free(clabel, st);
        if (s) dl_store_destroy(s);
        return rc;
    }
    s->unit = in->unit;
    s->nonneg = in->nonneg;
    s->clabel = clabel;
    *out = s;
    return DL_OK;
}
