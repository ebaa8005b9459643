// kernels.h -- launch interfaces of the library's kernels (host side).
#pragma once

#include <cuda.h>

#include "emit.cuh"
#include "internal.h"

namespace dl {

// ---- K2+K3+K5 tensor-core epsilon-join (join_tc.cu)
struct TcParams {
    const int4 *units;       // {m, nb, ne, 0}: R tile m against S tiles [nb, ne)
    int n_units;
    const int *n_units_dev;  // when not NULL the unit count is read here (units built on the device)
    const uint32_t *tile_mask;   // when not NULL: [R tiles][mask_ntw] bits; a unit's S tiles with a
    int mask_ntw;                // clear bit are skipped (the pruned join; one-SM tiles only)
    int nR, nS;
    int kc;                  // K chunks of 64 (dp / 64)
    int stages;              // S ring depth
    int a_slots;             // R-tile slots (2: the next unit's R tile loads during this one)
    int upper;               // 1: self-join, only columns c > r are pairs
    const float4 *rowpar;    // [m_tiles*128] {alpha_acc, alpha_rej, rq, nqt}
    const float *beta;       // S: RN32(||x||^2/2), +inf padding
    const float4 *cstat;     // S: per 32-column chunk {P1, P2, P3, min beta}
    float *dump_h;           // diagnostics: h of every pair [nR][nS] in caller order (NULL: off)
    float *dump_e;           // diagnostics: the bound E of every pair
    const int32_t *orig_r, *orig_s;   // diagnostics: caller row of each store row
    const float *sc_r;       // FP8: per-row power-of-two scales of R (NULL for BF16)
    const float *sc_s;       // FP8: per-32-row-chunk scales of S
    uint2 *cand;             // candidates: {r, c | 0x80000000 if a band pair, else a proven match}
    unsigned long long *cand_cnt;
    unsigned long long cand_cap;
    int *err;                // set to 1 when a bounded wait expired
    long long wait_budget;   // SM clocks an abortable pipeline wait may take (set by launch_tc_join)
    // top-k epilogue (units carry the S split in .w; state per (row, split, half) slot)
    int tk_k;                // k
    int tk_cap;              // candidate-list capacity per slot
    int tk_slots;            // slots per row (2 x splits)
    float *tk_heap;          // [rows][slots][k] min-heap of the k largest lower bounds of h
    uint2 *tk_list;          // [rows][slots][cap] {column, float bits of the upper bound of h}
    int *tk_cnt;             // [rows][slots] list fill
    float *tk_theta;         // [rows][slots] final threshold (heap minimum)
    unsigned *tk_row_theta;  // [rows] best threshold of any slot of the row (order-preserving encoding)
    int *tk_overflow;        // [rows] set when a list cannot hold every candidate
};

// Candidate entry flag: set for a band pair (needs the exact recheck).
constexpr uint32_t kBandFlag = 0x80000000u;

struct TcLaunch {
    const CUtensorMap *tmA, *tmB;
    TcParams p;
    int BN;
    int grid;           // CTAs (with cg2: twice the CTA pairs wanted; clamped to the resident pairs)
    bool cg2 = false;   // CTA pairs (tcgen05 cta_group::2) on 256-row tiles: units count 256-row tiles,
                        // tmB's box is BN/2 rows, rowpar covers the rows rounded up to 256
    bool wide = false;  // 16 epilogue warps (256-column epsilon-join); plan with tc_plan(..., wide)
};

// Shared-memory plan of the tensor-core kernel (wide: the 16-warp epilogue's layout).
// stream: a plan left with fewer than three stages beside one resident R tile streams the R
// tile's chunks with the S chunks instead (a_slots = 0; the one-SM epsilon-join only).
void tc_plan(int BN, int kc, int *stages, int *a_slots, bool fp8 = false, bool cg2 = false, bool wide = false,
             bool stream = false);
// Clock budget of the tensor-core kernels' abortable waits: the default (about 1 s),
// unless dl_debug_set_wait_budget set another.
long long tc_wait_budget();
// *grid_out (optional) receives the CTAs actually launched.
int launch_tc_join(const TcLaunch &L, cudaStream_t st, bool topk = false, bool fp8 = false, int *grid_out = nullptr);

// ---- K8 SIMT FP32 join (join_simt.cu)
struct SimtParams {
    const float *R;
    const float *S;
    int nR, nS, d;
    int upper;          // self-join: only c > r
    int tiles_m;        // filled by the launcher
    int exact;          // 0 plain, 1 exact (band output)
    int metric;         // 0 squared L2, 1 L1, 2 chi-square (distances compared with t_acc / t_rej)
    float t_acc, t_rej; // exact thresholds; plain uses t_acc only
    JoinOut out;
};
int launch_simt_join(SimtParams p, cudaStream_t st);
// Exact decision of the histogram-distance band pairs (metric 1 L1, 2 chi-square): the
// canonical FP64 distance compared with eps (recheck.cu).
int launch_hist_recheck(int metric, const uint2 *band, const unsigned long long *band_cnt, unsigned long long band_cap,
                        const float *R, const float *S, int d, double eps, const JoinOut &out,
                        unsigned long long *n_fp64, int grid, cudaStream_t st);

// ---- K6 recheck and small per-join kernels (recheck.cu)
int launch_recheck(const uint2 *band, const unsigned long long *band_cnt, unsigned long long band_cap, const float *R,
                   const float *S, int d, double e2, float t_acc, float t_rej, const JoinOut &out,
                   unsigned long long *n_fp64, int grid, cudaStream_t st);
int launch_rowpar(const double *nq64, const float4 *rowb, int64_t n, int64_t n_tot, int dp, double e2,
                  const double *row_e2, double g64, float4 *rowpar, cudaStream_t st, const float2 *rowb8 = nullptr);
// Turn the tensor-core kernel's candidate list into id pairs: proven matches are
// translated directly, band pairs are rechecked exactly first (recheck.cu).
int launch_finalize(const uint2 *cand, const unsigned long long *cand_cnt, unsigned long long cand_cap, const float *R,
                    const float *S, int d, double e2, float t_acc, float t_rej, const JoinOut &out,
                    unsigned long long *n_fp64, unsigned long long *n_band, int grid, cudaStream_t st, int nR, int nS);
// The inner-product join (recheck.cu): per-row thresholds for the tensor-core epilogue, and the
// exact decision of its candidates (FP32 dot with its bound, canonical FP64 dot if needed).
int launch_rowpar_ip(const float4 *rowb, int64_t n, int64_t n_tot, int dp, double t, float4 *rowpar, cudaStream_t st);
int launch_finalize_ip(const uint2 *cand, const unsigned long long *cand_cnt, unsigned long long cand_cap,
                       const float *R, const float *S, int d, double t, const JoinOut &out,
                       unsigned long long *n_fp64, unsigned long long *n_band, int grid, cudaStream_t st, int nR, int nS);
// Top-k under the L1 (metric 1) or chi-square (metric 2) distance (hist_topk.cu): outputs at
// the caller's query row order, [nQ][k] ids and canonical distances, -1 past the store.
int hist_topk(const dl_store *Q, const dl_store *S, int metric, int k, int64_t *out_ids, double *out_d,
              cudaStream_t st, dl_join_stats *stats);
int launch_diag(const int64_t *ids, int64_t n, int64_t *out_r, int64_t *out_s, unsigned long long *out_cnt,
                unsigned long long cap, cudaStream_t st);

// ---- top-k core (topk.cu): every row of Q against S, outputs at row_off or caller row * k
int topk_core(const dl_store *Q, const dl_store *S, int k, const int *row_k, const int64_t *row_off,
              int64_t *out_ids, double *out_d2, const dl_join_opts &o, cudaStream_t st, dl_join_stats *stats);

// Order-preserving encoding of a float as unsigned (larger float -> larger code),
// so that a running maximum can be kept with atomicMax.
__device__ __forceinline__ unsigned float_order_code(float f)
{
    const unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float float_from_order_code(unsigned c)
{
    return __uint_as_float((c & 0x80000000u) ? (c & 0x7fffffffu) : ~c);
}

}  // namespace dl
