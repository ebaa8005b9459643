/*
 * dl.h -- C ABI of the GB300 exact epsilon-similarity join and top-k join.
 *
 * The operation (Krishnan, Dziedzic, Elmore, "DeepLens: Towards a Visual Data
 * Management System", CIDR 2019):
 *   - Sec. 2.2: a patch is (ImgRef, Data, MetaData) where Data is a dense
 *     n-dimensional vector; here a patch is an opaque int64 id plus a float32
 *     feature row of length d (ImgRef and MetaData are not used by the join).
 *   - Sec. 5 "Nested Loop Join": compare every pair of patches from two
 *     collections and return the pairs that satisfy the predicate.
 *   - Sec. 3.2: the image-matching predicate thresholds feature similarity with
 *     a Euclidean distance threshold. Read here as
 *         D(q, x) = sum_k (q_k - x_k)^2  <=  eps^2      (inclusive)
 *     with D evaluated as the canonical FP64 sum: k ascending,
 *     t = (double)q_k - (double)x_k, s = s + t*t, round-to-nearest, no FMA.
 *     The returned pair set is exactly the set that evaluation selects.
 *   - Sec. 6.2 q1 (closest image to a query image): the top-k join, ordered by
 *     (canonical D, store row index).
 *
 * Conventions for every entry point:
 *   - Return an int status (dl_status); nothing throws across the ABI.
 *     dl_last_error() gives a thread-local message for the last failure.
 *   - Inputs are copied; the caller may free them when the call returns.
 *   - Stores and results are owned by the library until their destroy/free call.
 *   - A stream argument is a cudaStream_t passed as void*; NULL is the legacy
 *     default stream. Calls that return a count synchronise that stream.
 *   - Everything runs on the CUDA device current on the calling thread, which
 *     must be an sm_103 GPU (GB300); there is no CPU fallback: without a usable
 *     GPU every compute call fails with DL_ECUDA.
 */
#ifndef DL_H
#define DL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum dl_status {
    DL_OK = 0,
    DL_EINVAL = 1,        /* bad argument: null pointer, size, d, eps, k, non-finite feature ... */
    DL_ENOMEM = 2,        /* a device or pinned-host allocation failed */
    DL_EOVERFLOW = 3,     /* a fixed output capacity was too small; see dl_result_count */
    DL_EAGAIN = 4,        /* (server) request not finished yet */
    DL_ETIMEOUT = 5,      /* (server) poll timed out / a bounded device wait expired */
    DL_ECUDA = 6,         /* a CUDA runtime call or kernel failed */
    DL_ECANCELED = 7,     /* (server) request was cancelled */
    DL_ENOMEM_ADMIT = 8,  /* (server) request can never fit the memory budget */
    DL_EFAILED = 9,       /* (server) request failed; it may be resubmitted */
    DL_EUNSUPPORTED = 10  /* valid request this build does not serve (e.g. d too large for a precision) */
} dl_status;

typedef enum dl_metric {
    DL_METRIC_L2 = 0,     /* squared Euclidean distance compared with eps^2 (Sec. 3.2) */
    DL_METRIC_COSINE = 1, /* cosine similarity on stores made by dl_store_normalize: eps is the
                             threshold c in [-1, 1] and a pair matches iff the canonical D of
                             the normalized rows is <= fl64(2 - 2c) (cos >= c for unit rows) */
    DL_METRIC_L1 = 2,     /* histogram L1 distance: canonical FP64 sum_k |q_k - x_k| <= eps
                             (k ascending, every step rounded to nearest); epsilon- and top-k joins */
    DL_METRIC_CHI2 = 3,   /* chi-square histogram distance on non-negative features: canonical FP64
                             sum over bins with q_k + x_k > 0 of (q_k - x_k)^2 / (q_k + x_k) <= eps
                             (no factor 1/2); epsilon- and top-k joins */
    DL_METRIC_IP = 4      /* inner-product threshold on rows of any norm (Sec. 3.2 "threshold the
                             similarity"): a pair matches iff the canonical FP64 dot product
                             sum_k q_k x_k (k ascending, every addition rounded to nearest; the
                             products are exact) is >= eps; epsilon-join only */
} dl_metric;

typedef enum dl_precision {
    DL_PREC_AUTO = 0,       /* BF16 tensor-core path when d <= 512, else FP8 e4m3 (ε-join);
                               top-k: BF16 when d <= 512, else FP32 */
    DL_PREC_BF16 = 1,       /* -2 q.x on tcgen05 tensor cores in BF16, FP32 accumulate; exact result */
    DL_PREC_FP8E4M3 = 2,    /* as BF16 but FP8 e4m3 with power-of-two scales (per 32-row chunk of
                               each store); exact result */
    DL_PREC_FP32 = 3,       /* FP32 SIMT distances + bound + FP64 recheck; exact result */
    DL_PREC_FP32_PLAIN = 4  /* plain FP32 SIMT join D32 <= (float)(eps*eps): the comparison
                               baseline, NOT exact near the threshold */
} dl_precision;

typedef enum dl_memkind {
    DL_MEM_HOST = 0,      /* pointer is host memory (pageable or pinned) */
    DL_MEM_DEVICE = 1     /* pointer is device memory of the current device */
} dl_memkind;

typedef enum dl_self_mode {
    DL_SELF_UPPER = 0,    /* self-join returns unordered pairs (i, j) with row i < row j */
    DL_SELF_FULL = 1      /* self-join returns every ordered pair, diagonal included */
} dl_self_mode;

typedef struct dl_store dl_store;
typedef struct dl_result dl_result;
typedef struct dl_server dl_server;

typedef struct dl_join_opts {
    int32_t precision;      /* dl_precision */
    int32_t self_mode;      /* dl_self_mode; used when the second store is NULL */
    int64_t out_capacity;   /* 0: the library sizes the output and re-runs on overflow;
                               >0: fixed capacity, overflow returns DL_EOVERFLOW with the
                               required count available through dl_result_count */
    void *cuda_stream;      /* cudaStream_t the work is ordered on */
    int32_t tile_n;         /* 0: autotuned; else the tensor-core tile width (128 or 256) */
    int32_t timing;         /* 1: record CUDA events around each kernel (dl_result_stats) */
    int32_t prune;          /* 1: the exact pruned epsilon-join (tensor-core precisions, L2 and
                               cosine): tile pairs whose bounding balls lie farther apart than
                               eps are skipped; best on stores from dl_store_cluster */
    int32_t cta_pair;       /* tensor-core epsilon-join: 0 autotuned (with tile_n 0), 1 one SM per
                               128-row tile, 2 a pair of SMs per 256-row tile (tcgen05 cta_group::2,
                               tile_n 256 only); the result is the same set either way */
    int32_t epilogue_warps; /* tensor-core epsilon-join and top-k: 0 autotuned (with tile_n 0 and
                               cta_pair 0), 8, or 16 (tile_n 256 on one SM: four warps per SM
                               sub-partition, best when many pairs are candidates); the same result
                               either way */
} dl_join_opts;

/* Fill `o` with defaults: AUTO precision, upper self mode, auto capacity, NULL stream. */
void dl_join_opts_default(dl_join_opts *o);

/* ---------------------------------------------------------------------------------
 * Stores: the device-resident patch collection (Sec. 3.2 "materialize" / Sec. 4.1).
 * ------------------------------------------------------------------------------- */

/*
 * Create a store of n patches with int64 `ids` [n] and float32 `feats` [n][d]
 * (row-major, contiguous). `where` tells whether both pointers are host or
 * device memory; the data are copied, then one pass (K1) derives the per-row
 * norms, the BF16 copy and the error-bound statistics the join kernels use.
 * Requirements: 1 <= d <= 1024, 0 <= n < 2^31, every feature finite with
 * |x| <= 2^40 (else DL_EINVAL). Ids are opaque and may repeat. On success *out
 * owns device memory until dl_store_destroy. Ordered on `cuda_stream`; the
 * call synchronises it (to report validation errors).
 */
int dl_store_create(dl_store **out, const int64_t *ids, const float *feats, int64_t n, int32_t d,
                    int32_t where, void *cuda_stream);

/*
 * A new store holding the unit-normalized rows of `in`, for the cosine metric (a metric
 * beyond the paper's Euclidean queries): same ids and the same caller row order, row
 * x^ = fl32(x_k / n) with n = fl32(sqrt(sum_k x_k^2)), the sum in FP64 with k ascending and
 * every addition rounded to nearest. The normalized FP32 rows are the ground truth of every
 * cosine join on the new store. A row with a zero norm has no direction: DL_EINVAL and *out
 * stays NULL. `in` is unchanged and may be destroyed afterwards. cuda_stream as for
 * dl_store_create; the call returns when the new store is ready.
 */
int dl_store_normalize(const dl_store *in, dl_store **out, void *cuda_stream);

/*
 * A copy of `in` (same rows, ids and caller rows) in a clustered row order, for the pruned
 * join (opts.prune; Sec. 5 and Sec. 7.3: the on-the-fly index join). The rows are grouped by
 * `iters` iterations of k-means with `n_clusters` centres, started from store rows spread
 * pseudo-randomly (row c * 1000003 mod n for centre c); each assignment step is the exact top-1 join of the rows against the centres. The
 * order changes no join result, only how many tile pairs the pruned join can skip.
 * Synchronizes cuda_stream. DL_EINVAL for n_clusters < 1 or iters outside [0, 100].
 */
int dl_store_cluster(const dl_store *in, int32_t n_clusters, int32_t iters, dl_store **out, void *cuda_stream);

/* Free a store. Joins that use it must have completed. NULL is accepted. */
int dl_store_destroy(dl_store *s);

/* Number of rows and dimension of a store. */
int dl_store_shape(const dl_store *s, int64_t *n, int32_t *d);

/*
 * Colour-histogram transformer (Sec. 4.1 "Transformers": colour histogram features
 * for image matching), the producer of the stores' features.
 *   frames  device, uint8 [n_frames][H][W][3], interleaved RGB, row-major, 16-byte aligned;
 *   boxes   device, int32 [n_boxes][5] = {frame, x0, y0, x1, y1}: the half-open pixel
 *           rectangle [x0, x1) x [y0, y1) of that frame;
 *   br, bg, bb  bins per channel, each in [1, 256], d = br*bg*bb <= 1024;
 *   out     device, float32 [n_boxes][d], row-major (caller-owned);
 *   count_ms  host, may be NULL: receives the CUDA-event time of the pixel-counting kernel.
 * Channel value v falls in bin floor(v*b/256) of that channel; the joint bin is
 * (r_bin*bg + g_bin)*bb + b_bin; out = count / (pixels of the box), each a correctly
 * rounded FP32 division. Errors: DL_EINVAL for bad sizes or alignment and for any
 * invalid box (outside its frame, empty, or more than 2^24 pixels), in which case
 * out is unspecified. The call synchronizes cuda_stream to report invalid boxes.
 */
int dl_color_hist(const uint8_t *frames, int64_t n_frames, int32_t H, int32_t W, const int32_t *boxes,
                  int64_t n_boxes, int32_t br, int32_t bg, int32_t bb, float *out, float *count_ms,
                  void *cuda_stream);

/* ---------------------------------------------------------------------------------
 * q4 deduplication (Sec. 6.2 q4, Sec. 7.4.3 and Table 1).
 * ------------------------------------------------------------------------------- */

/*
 * Connected components of the graph on rows 0..n-1 whose edges are (pair_a[e], pair_b[e]),
 * e < m (device int64 arrays of row indices; self-loops and repeats allowed). label
 * (device int64 [n], caller-owned) receives, for every row, the smallest row index of its
 * component; *n_components (host, may be NULL) the number of components. n must be below
 * 2^31. DL_EINVAL when an edge names a row outside [0, n). Synchronizes cuda_stream.
 */
int dl_components(int64_t n, const int64_t *pair_a, const int64_t *pair_b, int64_t m, int64_t *label,
                  int64_t *n_components, void *cuda_stream);

typedef enum dl_dedup_plan {
    DL_DEDUP_ALL = 0,           /* components of the self-join of every row */
    DL_DEDUP_FILTER_MATCH = 1,  /* keep the rows labelled `target`, join them, count their components
                                   (Table 1 "Patch, Filter, Match"); other rows get component -1 */
    DL_DEDUP_MATCH_FILTER = 2   /* join every row, count the components holding at least one row
                                   labelled `target` (Table 1 "Patch, Match, Filter") */
} dl_dedup_plan;

/*
 * Count distinct objects (q4): the epsilon self-join of X (metric and eps as in
 * dl_sim_join; opts->self_mode and out_capacity are ignored), then its connected
 * components. labels: device int32 [n] per caller row (required by the two label plans).
 * comp: device int64 [n], per caller row the smallest caller row of its component (or -1,
 * see the plan). *n_distinct (host): the number of distinct objects under the plan.
 * Synchronizes opts->cuda_stream. Errors as dl_sim_join.
 */
int dl_dedup(const dl_store *X, int32_t metric, double eps, const int32_t *labels, int32_t target, int32_t plan,
             const dl_join_opts *opts, int64_t *comp, int64_t *n_distinct);

/* ---------------------------------------------------------------------------------
 * Joins.
 * ------------------------------------------------------------------------------- */

/*
 * Epsilon-similarity join (Sec. 5 nested-loop semantics, Sec. 3.2 predicate):
 * every pair (r in R, s in S) with canonical D(r, s) <= eps*eps, as id pairs.
 * S == NULL is a self-join of R, in opts->self_mode. eps must be >= 0 and not
 * NaN; eps = +inf returns every pair. With DL_METRIC_COSINE, eps is the cosine
 * threshold c in [-1, 1] and both stores must come from dl_store_normalize. With
 * DL_METRIC_L1 / DL_METRIC_CHI2 the predicate is the histogram distance <= eps; these
 * run with DL_PREC_FP32 (AUTO picks it) or DL_PREC_FP32_PLAIN (BF16 / FP8 give
 * DL_EUNSUPPORTED), and CHI2 gives DL_EINVAL when a feature is negative. With
 * DL_METRIC_IP, eps is the inner-product threshold t (any value but NaN; -inf returns
 * every pair, +inf none); it runs on the BF16 tensor-core path (AUTO picks it), for
 * R x S and the upper self mode, without pruning (FP32 / FP8 precisions, the full self
 * mode and opts->prune give DL_EUNSUPPORTED). opts may be
 * NULL (defaults). On success *out holds the result (free with
 * dl_result_free); on DL_EOVERFLOW *out is also set so that the required
 * count can be read. The pair order is unspecified (the result is a set).
 */
int dl_sim_join(const dl_store *R, const dl_store *S, int32_t metric, double eps,
                const dl_join_opts *opts, dl_result **out);

/*
 * Top-k join (Sec. 6.2 q1 generalised to k): for every row of Q, the min(k, |S|)
 * rows of S with the smallest canonical D, ordered by (D, S row index); ties
 * beyond the k-th are not returned. 1 <= k <= 1024. With DL_METRIC_COSINE (both
 * stores from dl_store_normalize) these are the k most similar rows, and the
 * distances returned are the canonical D of the normalized rows (2 - 2 cos). With
 * DL_METRIC_L1 / DL_METRIC_CHI2 (DL_PREC_AUTO or FP32; BF16 gives DL_EUNSUPPORTED,
 * negative features under chi-square DL_EINVAL) the rows with the smallest canonical
 * histogram distance, which is what the distances hold; DL_EOVERFLOW if more than
 * 8,192 columns of one row tie within the FP32 bound of its k-th distance.
 */
int dl_topk_join(const dl_store *Q, const dl_store *S, int32_t metric, int32_t k,
                 const dl_join_opts *opts, dl_result **out);

/*
 * Exact epsilon-join that allocates nothing (no counterpart in the paper; it
 * exists for callers that cannot allocate device memory when they join, e.g.
 * code running under a memory planner that owns the whole device or a
 * real-time loop that must not enter the allocator).
 * All pointers are DEVICE memory owned by the caller: R [nR][d] float32 and
 * r_ids [nR]; S [nS][d] and s_ids [nS], or S == NULL for a self-join of R in
 * `self_mode`; out_r / out_s receive up to out_cap id pairs. *n_out (host)
 * receives the number of matching pairs. The result is the same set
 * dl_sim_join returns (exact FP32 path: FP32 distances with an error bound,
 * FP64 recheck of the undecided pairs).
 * Preconditions, each refused with DL_EINVAL: R and S 16-byte aligned when
 * d % 4 == 0 (else 4-byte), ids and outputs 8-byte aligned (checked before any
 * launch); every feature finite with |x| <= 2^40, the domain dl_store_create
 * also enforces (checked on the device; the outputs are then unspecified).
 * Working memory is a 512 KiB static device array in the library, held by every
 * GPU that loads it until exit; it holds at most 65,536 pairs inside the FP32
 * error band of eps^2. A call that needs more returns DL_EOVERFLOW (outputs
 * incomplete); more than out_cap matches also returns DL_EOVERFLOW with the
 * required count in *n_out. The first call on each device looks up the
 * array's device address, so make that first call before any stream capture.
 * Every call shares the one array: calls whose work overlaps on the GPU
 * (other streams, other host threads) race and must not be issued. The call
 * synchronises `cuda_stream`.
 */
int dl_sim_join_noalloc(const float *R, const int64_t *r_ids, int64_t nR, const float *S,
                        const int64_t *s_ids, int64_t nS, int32_t d, double eps, int32_t self_mode,
                        int64_t *out_r, int64_t *out_s, int64_t out_cap, int64_t *n_out,
                        void *cuda_stream);

/*
 * Diagnostics for the error bound of the low-precision stage (no counterpart in
 * the paper). Runs the tensor-core pass of an R x S join in `precision`
 * (DL_PREC_BF16 or DL_PREC_FP8E4M3) and writes, for every pair at the callers'
 * row order, the kernel's approximation h~ of h = q.x - ||x||^2/2 (so that
 * D = ||q||^2 - 2h) into h_out[|R|][|S|] and the bound E it uses into
 * e_out[|R|][|S|] (device memory, caller-owned). |R| |S| <= 2^28. A sound kernel
 * has |h~ - h| <= E for every pair.
 */
int dl_debug_scores(const dl_store *R, const dl_store *S, int32_t precision, float *h_out, float *e_out,
                    void *cuda_stream);

/*
 * Diagnostics for failure detection (no counterpart in the paper). Every
 * pipeline wait inside the tensor-core kernels is bounded: past its budget the
 * kernel raises an abort flag, lets its copies in flight land, finishes its
 * issued MMAs, frees its tensor memory and returns, and the calling entry point
 * reports DL_ETIMEOUT (a server marks the batch's requests DL_EFAILED). This
 * sets that budget, in SM clocks, for every tensor-core kernel launched after
 * the call on any thread; 0 restores the default of 2e9 clocks (about 1 s).
 * A budget below 64 clocks makes every abortable wait expire at once, so a
 * healthy join times out deterministically; this is how the tests drive the
 * abort path without faulting or hanging a GPU. Returns DL_EINVAL for
 * clocks < 0.
 */
int dl_debug_set_wait_budget(int64_t clocks);

/*
 * Diagnostics of the bounds-checked build (no counterpart in the paper). A
 * library compiled with -DDL_CHECKED (paper_1812_07607_gb300.build with
 * checked=True: libdlsimjoin_checked.so) guards computed shared- and global-
 * memory indices of its hot kernels; a failed check skips the access (nothing
 * traps) and records the first failure per translation unit as
 * (site << 40) | (index & (2^40 - 1)). dl_debug_check_word stores the first
 * recorded failure in *word (0: none) and clears the records; in the normal
 * build it always stores 0. dl_debug_check_selftest records a failure of site 99
 * with `index` on purpose (a check of a constant-false condition guarding no
 * access) so a test can see the mechanism work; it returns DL_EUNSUPPORTED in
 * the normal build.
 */
int dl_debug_check_word(uint64_t *word);
int dl_debug_check_selftest(int64_t index);

/* ---------------------------------------------------------------------------------
 * Batches: many epsilon-join and top-k requests against one resident store.
 * ------------------------------------------------------------------------------- */

typedef enum dl_request_kind {
    DL_REQ_EPS = 0,       /* epsilon-join of the request's query rows against the store */
    DL_REQ_TOPK = 1       /* top-k join of the request's query rows against the store */
} dl_request_kind;

typedef struct dl_request {
    int32_t kind;         /* dl_request_kind */
    int32_t k;            /* DL_REQ_TOPK: 1..1024 */
    double eps;           /* DL_REQ_EPS: >= 0, not NaN */
    int64_t q_begin;      /* first row of this request in the batch's query arrays */
    int64_t nq;           /* number of query rows (>= 0) */
} dl_request;

/*
 * Run n_req requests of uneven sizes as one batch against the store S (the
 * paper's image-matching queries, Sec. 6.2 q1/q4, issued many at a time).
 * q_ids [nq_total] and q_feats [nq_total][d] hold every request's query rows;
 * request i uses rows [q_begin, q_begin + nq) (ranges may overlap). `where`
 * tells whether both are host or device memory; they are copied. All
 * epsilon-join rows run in one persistent tensor-core launch (each row with its
 * request's eps), all top-k rows in another (each row with its request's k),
 * then the outputs are routed per request. Each request's result is the set (or
 * ordered list) the single-request call would return. On success *out holds a
 * batch result; read it with dl_result_request_pairs / dl_result_request_topk.
 */
int dl_batch_join(const dl_store *S, const int64_t *q_ids, const float *q_feats, int64_t nq_total, int32_t d,
                  int32_t where, const dl_request *reqs, int32_t n_req, const dl_join_opts *opts,
                  dl_result **out);

/* Pairs of epsilon-join request `req` of a batch result (same conventions as dl_result_pairs). */
int dl_result_request_pairs(dl_result *r, int32_t req, int32_t where, const int64_t **r_ids,
                            const int64_t **s_ids, int64_t *n);

/* Top-k rows of top-k request `req` of a batch result (same conventions as dl_result_topk). */
int dl_result_request_topk(dl_result *r, int32_t req, int32_t where, const int64_t **ids,
                           const double **dist2, int32_t *k, int64_t *nq);

/* ---------------------------------------------------------------------------------
 * Serving: a request loop with continuous batching over a resident store.
 * ------------------------------------------------------------------------------- */

typedef struct dl_server_stats {
    int64_t completed;            /* requests finished */
    int64_t failed;               /* requests whose batch failed (resubmittable) */
    int64_t batches;              /* batches launched */
    int64_t queued;               /* requests waiting for a slot */
    int32_t in_flight_batches;    /* batches on the GPU now */
    int64_t admission_waits;      /* times the head request waited for memory */
    double p50_ms, p99_ms, max_ms, mean_ms;   /* submit-to-ready latency of completed requests */
    double mean_batch_requests;   /* requests per batch */
} dl_server_stats;

/*
 * Start a request loop over store S (kept resident; it must outlive the server).
 * Up to `slots` batches (1..8) run at once, each on its own CUDA stream, so work
 * of consecutive batches overlaps on the device. A batch takes queued requests
 * in arrival order up to `max_batch_rows` query rows and as long as their memory
 * estimate fits both `mem_budget_bytes` minus what is in flight and the
 * device's free memory. The paper has no serving layer; this serves its
 * image-matching queries (Sec. 6.2) arriving one by one.
 */
int dl_server_create(dl_server **out, const dl_store *S, int64_t mem_budget_bytes, int32_t slots,
                     int64_t max_batch_rows, const dl_join_opts *opts);

/*
 * Queue one request: nq query rows (host memory, copied) and either an
 * epsilon-join (kind DL_REQ_EPS, eps) or a top-k join (DL_REQ_TOPK, k). Returns
 * a ticket. DL_ENOMEM_ADMIT if the request could never fit the budget or the
 * batch row limit.
 */
int dl_submit(dl_server *sv, const int64_t *q_ids, const float *q_feats, int64_t nq, int32_t kind, double eps,
              int32_t k, uint64_t *ticket);

/*
 * Result of a ticket: DL_OK with *out set (a single-request result, free with
 * dl_result_free); DL_EAGAIN if not ready and timeout_us == 0; DL_ETIMEOUT if
 * not ready after waiting timeout_us; DL_ECANCELED; DL_EFAILED (resubmit). A
 * ticket is consumed by the call that returns its final status.
 */
int dl_poll(dl_server *sv, uint64_t ticket, int64_t timeout_us, dl_result **out);

/* Cancel a request that is still queued (DL_EAGAIN if it is already running). */
int dl_cancel(dl_server *sv, uint64_t ticket);

/* Latency and batching statistics. */
int dl_server_get_stats(dl_server *sv, dl_server_stats *st);

/* Stop the loop: queued requests are dropped, running batches finish first. */
int dl_server_destroy(dl_server *sv);

/* ---------------------------------------------------------------------------------
 * Results.
 * ------------------------------------------------------------------------------- */

/* Number of pairs of an epsilon-join result (also valid after DL_EOVERFLOW). */
int dl_result_count(const dl_result *r, int64_t *n);

/*
 * Pair ids of an epsilon-join result: r_ids[i], s_ids[i] for i < *n. With
 * where == DL_MEM_DEVICE the pointers are device memory owned by the result;
 * with DL_MEM_HOST the first call copies them into result-owned host memory.
 */
int dl_result_pairs(dl_result *r, int32_t where, const int64_t **r_ids, const int64_t **s_ids,
                    int64_t *n);

/*
 * Top-k result: ids[nq][k] (int64) and dist2[nq][k] (double, the canonical D).
 * Slots past min(k, |S|) hold id -1 and dist2 -1.0. `where` as for dl_result_pairs.
 */
int dl_result_topk(dl_result *r, int32_t where, const int64_t **ids, const double **dist2,
                   int32_t *k, int64_t *nq);

typedef struct dl_join_stats {
    int64_t pairs_evaluated;    /* pairs the join is defined over (|R||S| or N(N-1)/2) */
    int64_t pairs_out;          /* pairs returned */
    int64_t band_pairs;         /* pairs whose low-precision distance was within the bound of eps */
    int64_t fp64_pairs;         /* band pairs the FP32 recheck could not decide (FP64 evaluated) */
    int64_t reruns;             /* times the call re-ran after growing an internal buffer */
    int32_t precision;          /* dl_precision actually used */
    int32_t tile_n;             /* tensor-core tile width used (0 for SIMT paths) */
    float ms_main;              /* device time of the main join kernel (opts.timing) */
    float ms_recheck;           /* device time of the recheck kernel (opts.timing) */
    float ms_total;             /* device time of all kernels of the call (opts.timing) */
    int32_t kernels_launched;   /* kernels this call launched */
    int64_t tile_pairs;         /* opts.prune: tile pairs of the join (0 without pruning) */
    int64_t tile_pairs_kept;    /* opts.prune: tile pairs that survived the ball test */
    int32_t cta_pair;           /* 2 when the tensor-core pass ran on SM pairs, else 1 (0 for SIMT paths) */
    int32_t grid_ctas;          /* CTAs of the (last) tensor-core launch: resident SMs it occupied */
    int32_t epilogue_warps;     /* epilogue warps of the tensor-core pass (0 for SIMT paths) */
} dl_join_stats;

int dl_result_stats(const dl_result *r, dl_join_stats *st);

/* Free a result (NULL accepted). */
int dl_result_free(dl_result *r);

/* ---------------------------------------------------------------------------------
 * Library.
 * ------------------------------------------------------------------------------- */

/* Thread-local description of the last failure on this thread ("" if none). */
const char *dl_last_error(void);

/* Library version string. */
const char *dl_version(void);

/* Total kernels this library has launched in this process (for launch accounting). */
int64_t dl_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* DL_H */
