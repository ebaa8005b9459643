// internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "dl.h"

struct dl_store;

namespace dl {

// ---------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
void clear_error();
int cuda_fail(cudaError_t e, const char *what);

#define DL_CUDA_TRY(expr)                                      \
    do {                                                       \
        cudaError_t _e = (expr);                               \
        if (_e != cudaSuccess) return ::dl::cuda_fail(_e, #expr); \
    } while (0)

// A scoped NVTX range: names an entry point or a stage on the Nsight Systems timeline
// (header-only NVTX; without a tool attached the push and pop do nothing).
struct NvtxScope {
    explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope &) = delete;
    NvtxScope &operator=(const NvtxScope &) = delete;
};

extern std::atomic<int64_t> g_launches;
inline void count_launch(int n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// ---------------------------------------------------------------- numeric constants
// Unit roundoff of FP32 / FP64 (round to nearest).
constexpr double kU32 = 5.9604644775390625e-08;   // 2^-24
constexpr double kU64 = 1.1102230246251565e-16;   // 2^-53

// Relative bound of the canonical FP64 distance sum against the exact real
// value: |D64 - D| <= (d+3) 2^-53 D (the oracle's first pin checks the same
// bound); one extra unit of margin.
inline double gamma64(int d) { return (d + 4) * kU64; }

// Relative bound of any FP32 evaluation of sum_k (q_k - x_k)^2 the library
// performs (sequential FMA chain, or lane partial sums plus a 5-level shuffle
// tree): (d + 8) 2^-24.
inline double gamma32(int d) { return (d + 8) * kU32; }

// Assumed relative bound of the tensor-core FP32 accumulation of d BF16 x BF16
// products (the products are exact in FP32; summation order and rounding of the
// hardware adder are not documented): d * 2^-20, sixteen times the textbook
// d * 2^-24. Checked empirically by the bound-validity test.
inline double gamma_tc(int dp) { return dp * 9.5367431640625e-07; }

// Absolute slack covering underflow/flush of tiny products.
inline double abs_slack_tc(int dp) { return dp * 8.271806125530277e-25; }   // dp * 2^-80

// ---------------------------------------------------------------- store
struct TmapCache {
    bool valid = false;
    int box_rows = 0;
    CUtensorMap map;
};

struct Store {
    int64_t n = 0;
    int32_t d = 0;
    int32_t dp = 0;          // d rounded up to a multiple of 64 (BF16 copy row length)
    int64_t n_pad = 0;       // n rounded up to a multiple of 256 (column-side padding)
    int device = 0;
    int64_t *ids = nullptr;  // [n] ids, in store order
    int32_t *orig = nullptr; // [n] caller's row index of each store row (rows are kept in norm order)
    float *x32 = nullptr;    // [n][d] FP32 master copy, in store order
    __nv_bfloat16 *xb = nullptr;  // [n][dp] BF16 copy, zero padded
    double *nq64 = nullptr;  // [n] sum of squares in FP64
    float *beta = nullptr;   // [n_pad] RN32(nq64 / 2); +inf in padding
    float4 *rowb = nullptr;  // [n] {||x - x~|| up, ||x~|| up, ||x|| up, |beta - ||x||^2/2| up}
    float4 *cstat = nullptr; // [n_pad / 32] per 32-row chunk {P1, P2, P3, min beta} of the BF16 bound
    TmapCache tmaps[3];      // BF16 boxes, cached per box height
    // FP8 e4m3 copy (built on the first FP8 join): row i is s_i * e4m3 codes, s_i a power of two
    int32_t dp8 = 0;         // d rounded up to a multiple of 128 (one 128-byte swizzle row per K chunk)
    void *fp8_block = nullptr;
    uint8_t *x8 = nullptr;   // [n][dp8] e4m3 codes of x / s
    float *sc8 = nullptr;    // [n_pad] s of each row: its 32-row chunk's scale (1 in padding)
    float *scc8 = nullptr;   // [n_pad/32] the chunk scales (power of two)
    float2 *rowb8 = nullptr; // [n] {||x - s x8|| up, ||s x8|| up}
    float4 *cstat8 = nullptr;// [n_pad/32] {P1, P2 (FP8), P3, beta_min}
    void *ip_block = nullptr;   // inner-product joins (built on first use): the column term
    float *beta_ip = nullptr;   // [n_pad] 0 (the dot product has no column term); +inf in padding
    float4 *cstat_ip = nullptr; // [n_pad / 32] chunk stats {P1, P2, P3, min beta_ip} for that term
    TmapCache tmaps8[3];     // FP8 boxes
    struct BallCache {       // bounding balls of the pruned join's tiles, per tile height
        int rows = 0;
        void *blk = nullptr;
        const float *centre = nullptr;   // [kMaxSeg][d][tiles]: ball u's centre coordinate k of each tile
        const float *radius = nullptr;   // [tiles][kMaxSeg]
        const int *nseg = nullptr;       // [tiles] balls of each tile
    } balls[2];
    std::mutex mu;           // guards tmaps and hints
    float nq_max = 0.f;      // largest ||x||^2 of the store (FP32 sum; used only inside slack terms)
    int64_t hint_pairs = 0;  // last output size seen with this store as R (capacity hint)
    int64_t hint_band = 0;
    double hint_batch_rate = 0.0;   // batch calls: candidates per evaluated pair last seen against this store
    bool unit = false;       // rows are the unit-normalized rows of another store (cosine metric)
    int nonneg = 0;          // 0 not checked yet, 1 every feature >= 0, 2 some feature < 0 (chi-square)
    int32_t *clabel = nullptr;   // [n] cluster of each store row (stores from dl_store_cluster), else NULL
};

// Create a store; gather == NULL orders rows by norm, else store row i is caller row gather[i].
int store_create_impl(dl_store **out, const int64_t *ids, const float *feats, int64_t n, int32_t d, int32_t where,
                      void *cuda_stream, const int32_t *gather);

// Whether every feature of the store is >= 0 (checked once, on first use, then cached).
int store_nonneg(Store *s, cudaStream_t st, bool *ok);

// The epsilon-join behind dl_sim_join; emit_ids (self-join only, device, [n] in store order)
// replaces the ids written to the output when not NULL.
int sim_join_impl(const dl_store *R, const dl_store *S, int32_t metric, double eps, const dl_join_opts *opts,
                  dl_result **out, const int64_t *emit_ids);

// Work units of the pruned join, built on the device with no host round trip (prune.cu): the
// ball test's tile mask (bit t of R tile m's row: S tile t may hold a pair within eps) and one
// unit {m, first, last + 1, 0} per (R tile, 64-tile S block) with a surviving tile, in the
// dense join's S-range-major order; the tensor-core kernel skips the masked-out tiles inside
// a unit. Everything lives in `block` (dev_alloc), freed by the caller after the join.
struct PruneUnits {
    void *block = nullptr;
    const int4 *units = nullptr;          // [cap]
    int cap = 0;                          // upper bound of the unit count (sizes the grid)
    const int *count = nullptr;           // device: units written
    const uint32_t *mask = nullptr;       // device: [R tiles][ntw]
    int ntw = 0;
    unsigned long long *kept = nullptr;   // device: surviving tile pairs
    int64_t total = 0;                    // tile pairs of the dense join
};
int prune_units(const dl_store *R, const dl_store *S, bool upper, int BN, double e2, cudaStream_t st, PruneUnits *pu);

// Build (or fetch from the store's cache) a 2-D BF16 tensor map over the store's
// BF16 copy with a box of 64 columns x box_rows rows and the 128-byte swizzle.
int get_tmap(Store *s, int box_rows, const CUtensorMap **out);

// FP8 copy of a store (built once, on first use) and its tensor maps (128-byte rows).
int ensure_fp8(Store *s, cudaStream_t st);
// Column arrays of the inner-product join (built once, on first use): beta_ip and cstat_ip.
int ensure_ip(Store *s, cudaStream_t st);
int get_tmap8(Store *s, int box_rows, const CUtensorMap **out);

// Assumed bound of the tensor-core accumulation of dp8 e4m3 x e4m3 products: dp8 * 2^-20,
// the same sixteen-times-textbook margin as BF16 (the measured FP8 accumulation error is
// below 0.02 FP32 ulps per term; the bound-validity test checks it).
inline double gamma_tc8(int dp8) { return dp8 * 9.5367431640625e-07; }

// ---------------------------------------------------------------- device pools
// Stream-ordered allocation from the current device's default memory pool.
int dev_alloc(void **p, size_t bytes, cudaStream_t st);
void dev_free(void *p, cudaStream_t st);

int device_sm_count();

// Autotuned tensor-core configuration: a tile width, plus kTunePair for SM-pair tiles or
// kTuneWide for the 16-warp epilogue.
constexpr int kTunePair = 1 << 12;
constexpr int kTuneWide = 1 << 13;
enum TuneKind { kTuneEpsRxS = 0, kTuneEpsSelf = 1, kTuneTopk = 2, kTuneEpsRxS8 = 3, kTuneEpsSelf8 = 4, kTuneBatch = 5 };
inline int tune_bn(int code) { return code & 0xfff; }
inline bool tune_pair(int code) { return (code & kTunePair) != 0; }
inline bool tune_wide(int code) { return (code & kTuneWide) != 0; }
int tune_pick(int dp, int kind, int64_t nR, int64_t nS, bool *trial);
void tune_record(int dp, int kind, int64_t nR, int64_t nS, int code, double kernel_ms, double pairs);
int tune_trials(int kind);   // calls of a shape class before it is decided

// Host-side directed conversions FP64 -> FP32 (the default conversion rounds to nearest).
inline float f32_ru(double x)
{
    float f = (float)x;
    if ((double)f < x) f = nextafterf(f, __builtin_inff());
    return f;
}
inline float f32_rd(double x)
{
    float f = (float)x;
    if ((double)f > x) f = nextafterf(f, -__builtin_inff());
    return f;
}

}  // namespace dl

struct dl_store : public dl::Store {};

struct dl_result {
    int kind = 0;             // 0 pairs, 1 topk, 2 batch (both, per request)
    int device = 0;
    cudaStream_t stream = nullptr;
    int64_t count = 0;        // pairs (kind 0)
    int64_t cap = 0;
    int64_t *d_r = nullptr, *d_s = nullptr;   // device pair ids
    int64_t *h_r = nullptr, *h_s = nullptr;   // host copies (pinned)
    int32_t k = 0;
    int64_t nq = 0;
    int64_t *d_ids = nullptr; double *d_d2 = nullptr;
    int64_t *h_ids = nullptr; double *h_d2 = nullptr;
    size_t h_bytes = 0;       // size of the pinned host block (h_r or h_ids)
    dl_join_stats stats{};
    // batch results: request i's pairs are [pair_off[i], pair_off[i+1]) of d_r/d_s, its top-k
    // rows are [topk_off[i], topk_off[i] + req_nq[i] * req_k[i]) of d_ids/d_d2
    std::vector<int32_t> req_kind, req_k;
    std::vector<int64_t> req_nq, pair_off, topk_off;
    int64_t n_topk_slots = 0;
    void *batch_block = nullptr;          // device block holding every batch output
    void *h_batch = nullptr;              // pinned host copy of batch_block (lazy)
    size_t batch_bytes = 0, h_batch_bytes = 0;
};
