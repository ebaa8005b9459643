/*
 * oracle.c -- TEST INFRASTRUCTURE, NOT THE PRODUCT.
 *
 * A plain, single-threaded, FP64 CPU statement of what the epsilon-similarity
 * join and its top-k variant compute. Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it. It shares no code, header or
 * constant with the CUDA library.
 *
 * What the paper fixes:
 *   - Sec. 5 "Nested Loop Join": the join compares every pair of patches from
 *     the two collections and returns the pairs that satisfy the predicate.
 *   - Sec. 3.2 "Derived Data": the predicate for image matching compares the
 *     features of two images and thresholds their similarity; the index the
 *     paper uses answers Euclidean threshold queries. So the predicate is an
 *     L2 distance threshold.
 *   - Sec. 6.2 q1: nearest image to a query image, i.e. the top-k join with k=1.
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   - compare the squared distance with eps*eps (no square root);
 *   - the threshold is inclusive (D <= eps^2);
 *   - a self-join returns unordered pairs i<j by default, or all ordered pairs
 *     including the diagonal in "full" mode;
 *   - top-k ties are broken by the smaller row index of the store side;
 *   - "exact" means the canonical FP64 value below: for k = 0..d-1 ascending,
 *     t = (double)q_k - (double)x_k, s = s + t*t, each operation rounded to
 *     nearest, no fused multiply-add (build with -ffp-contract=off);
 *   - cosine similarity (a further metric; the paper names only Euclidean
 *     queries) is taken on unit-normalized rows: n = fl32(sqrt(sum_k x_k^2)),
 *     the sum in FP64 with k ascending, x^_k = fl32(x_k / n); a pair matches
 *     iff the canonical D(q^, x^) <= fl64(2 - 2c), the L2 form of cos >= c for
 *     unit vectors. Rows with a zero norm have no direction and are rejected.
 *   - L1 and chi-square histogram distances (the other further metrics): for
 *     k ascending, t = (double)q_k - (double)x_k, s = s + |t| (L1), or
 *     u = (double)q_k + (double)x_k and, where u > 0, s = s + (t*t)/u
 *     (chi-square, no factor 1/2); every operation rounded to nearest. A pair
 *     matches iff s <= eps (these distances are not squared); their top-k orders
 *     by (distance, store row) as the L2 top-k does.
 *   - inner-product threshold (the general form of the cosine metric on rows of
 *     any norm): the canonical dot product s = s + (double)q_k * (double)x_k, k
 *     ascending, each step rounded to nearest (the FP64 products of two floats are
 *     exact); a pair matches iff s >= t.
 *   - colour histograms (Sec. 4.1 transformers): a patch is a box of a frame of
 *     8-bit interleaved RGB pixels; channel value v falls in bin floor(v*b/256)
 *     of its channel's b bins, the joint bin is (r*bg + g)*bb + b, and the
 *     histogram is count / (pixels in the box), one FP32 division per bin.
 *   - q4 deduplication (Sec. 6.2 q4, Sec. 7.4.3): the distinct objects are the
 *     connected components of the self-join's pairs; each row is labelled with
 *     the smallest row index of its component.
 *
 * Parity pins (tests/test_oracle_pins.py): exact rational brute force, integer
 * grid and one-hot closed forms, symmetry, zero self-distance, monotonicity in
 * eps, union and permutation laws, top-k/join consistency, and a mutation test
 * that plants mistakes in a copy of this file.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Canonical squared Euclidean distance (the definition of "exact"). */
double oracle_sqdist(const float *q, const float *x, int32_t d)
{
    double s = 0.0;
    for (int32_t k = 0; k < d; ++k) {
        double t = (double)q[k] - (double)x[k];
        s = s + t * t;
    }
    return s;
}

/*
 * Nested-loop epsilon-join (Sec. 5).
 *   mode 0: R x S, every (i, j).
 *   mode 1: self-join of R, unordered pairs i < j.
 *   mode 2: self-join of R, every ordered (i, j) including i == j.
 * Writes up to `cap` row-index pairs and returns the number of matching pairs.
 */
int64_t oracle_join(const float *R, int64_t nR, const float *S, int64_t nS, int32_t d,
                    double eps, int32_t mode, int64_t *out_r, int64_t *out_s, int64_t cap)
{
    const double e2 = eps * eps;
    const float *T = (mode == 0) ? S : R;
    const int64_t nT = (mode == 0) ? nS : nR;
    int64_t cnt = 0;
    for (int64_t i = 0; i < nR; ++i) {
        int64_t j0 = (mode == 1) ? i + 1 : 0;
        for (int64_t j = j0; j < nT; ++j) {
            double s = oracle_sqdist(R + i * (int64_t)d, T + j * (int64_t)d, d);
            if (s <= e2) {
                if (cnt < cap) {
                    out_r[cnt] = i;
                    out_s[cnt] = j;
                }
                ++cnt;
            }
        }
    }
    return cnt;
}

/* Canonical distances of rows [r0, r1) of R against every row of S, row-major. */
void oracle_dist_block(const float *R, int64_t r0, int64_t r1, const float *S, int64_t nS,
                       int32_t d, double *out)
{
    for (int64_t i = r0; i < r1; ++i)
        for (int64_t j = 0; j < nS; ++j)
            out[(i - r0) * nS + j] = oracle_sqdist(R + i * (int64_t)d, S + j * (int64_t)d, d);
}

typedef struct {
    double d2;
    int64_t j;
} oracle_cand;

static int cand_cmp(const void *a, const void *b)
{
    const oracle_cand *x = (const oracle_cand *)a, *y = (const oracle_cand *)b;
    if (x->d2 < y->d2) return -1;
    if (x->d2 > y->d2) return 1;
    return (x->j < y->j) ? -1 : (x->j > y->j);
}

/*
 * Top-k join (Sec. 6.2 q1 generalised to k): for every query row, all store rows
 * ordered by (canonical distance, store row index), first min(k, nS) kept.
 * out_idx / out_d2 are [nQ][k]; entries past min(k, nS) are set to -1 / -1.0.
 * Returns 0, or -1 when the scratch allocation fails.
 */
int32_t oracle_topk(const float *Q, int64_t nQ, const float *S, int64_t nS, int32_t d, int32_t k,
                    int64_t *out_idx, double *out_d2)
{
    oracle_cand *c = (oracle_cand *)malloc(sizeof(oracle_cand) * (size_t)(nS > 0 ? nS : 1));
    if (!c) return -1;
    int64_t keep = (k < nS) ? k : nS;
    for (int64_t i = 0; i < nQ; ++i) {
        for (int64_t j = 0; j < nS; ++j) {
            c[j].d2 = oracle_sqdist(Q + i * (int64_t)d, S + j * (int64_t)d, d);
            c[j].j = j;
        }
        qsort(c, (size_t)nS, sizeof(oracle_cand), cand_cmp);
        for (int64_t t = 0; t < k; ++t) {
            out_idx[i * k + t] = (t < keep) ? c[t].j : -1;
            out_d2[i * k + t] = (t < keep) ? c[t].d2 : -1.0;
        }
    }
    free(c);
    return 0;
}

/*
 * Unit-normalized copy of X [n][d] (the cosine metric's rows): n_i =
 * fl32(sqrt(sum_k x_k^2)) with the sum in FP64, k ascending, each step rounded
 * to nearest; out_k = fl32(x_k / n_i). Returns the number of rows with a zero
 * norm (their output row is left zero).
 */
int64_t oracle_normalize(const float *X, int64_t n, int32_t d, float *out)
{
    int64_t bad = 0;
    for (int64_t i = 0; i < n; ++i) {
        const float *x = X + i * (int64_t)d;
        float *o = out + i * (int64_t)d;
        double s = 0.0;
        for (int32_t k = 0; k < d; ++k) s = s + (double)x[k] * (double)x[k];
        const float nr = (float)sqrt(s);
        if (!(nr > 0.0f)) {
            ++bad;
            for (int32_t k = 0; k < d; ++k) o[k] = 0.0f;
            continue;
        }
        for (int32_t k = 0; k < d; ++k) o[k] = x[k] / nr;
    }
    return bad;
}

/*
 * Cosine-similarity join on normalized rows: the nested loop of oracle_join with
 * the predicate canonical D(q^, x^) <= fl64(2 - 2c).
 */
int64_t oracle_cosine_join(const float *Rn, int64_t nR, const float *Sn, int64_t nS, int32_t d,
                           double c, int32_t mode, int64_t *out_r, int64_t *out_s, int64_t cap)
{
    const double e2 = 2.0 - 2.0 * c;
    const float *T = (mode == 0) ? Sn : Rn;
    const int64_t nT = (mode == 0) ? nS : nR;
    int64_t cnt = 0;
    for (int64_t i = 0; i < nR; ++i) {
        int64_t j0 = (mode == 1) ? i + 1 : 0;
        for (int64_t j = j0; j < nT; ++j) {
            double s = oracle_sqdist(Rn + i * (int64_t)d, T + j * (int64_t)d, d);
            if (s <= e2) {
                if (cnt < cap) {
                    out_r[cnt] = i;
                    out_s[cnt] = j;
                }
                ++cnt;
            }
        }
    }
    return cnt;
}

/* Canonical L1 distance: k ascending, FP64, each operation rounded to nearest. */
double oracle_l1dist(const float *q, const float *x, int32_t d)
{
    double s = 0.0;
    for (int32_t k = 0; k < d; ++k) {
        double t = (double)q[k] - (double)x[k];
        s = s + fabs(t);
    }
    return s;
}

/* Canonical chi-square distance sum_k (q_k - x_k)^2 / (q_k + x_k); bins with q_k + x_k == 0 add nothing. */
double oracle_chi2dist(const float *q, const float *x, int32_t d)
{
    double s = 0.0;
    for (int32_t k = 0; k < d; ++k) {
        double t = (double)q[k] - (double)x[k];
        double u = (double)q[k] + (double)x[k];
        if (u > 0.0) s = s + (t * t) / u;
    }
    return s;
}

/*
 * Nested-loop join with a histogram distance: metric 1 = L1, 2 = chi-square;
 * a pair matches iff its distance <= eps. Modes and output as in oracle_join.
 */
int64_t oracle_hist_join(const float *R, int64_t nR, const float *S, int64_t nS, int32_t d, int32_t metric,
                         double eps, int32_t mode, int64_t *out_r, int64_t *out_s, int64_t cap)
{
    const float *T = (mode == 0) ? S : R;
    const int64_t nT = (mode == 0) ? nS : nR;
    int64_t cnt = 0;
    for (int64_t i = 0; i < nR; ++i) {
        int64_t j0 = (mode == 1) ? i + 1 : 0;
        for (int64_t j = j0; j < nT; ++j) {
            const float *q = R + i * (int64_t)d, *x = T + j * (int64_t)d;
            double s = (metric == 1) ? oracle_l1dist(q, x, d) : oracle_chi2dist(q, x, d);
            if (s <= eps) {
                if (cnt < cap) {
                    out_r[cnt] = i;
                    out_s[cnt] = j;
                }
                ++cnt;
            }
        }
    }
    return cnt;
}

/* Histogram distances of rows [r0, r1) of R against every row of S, row-major. */
void oracle_hist_dist_block(const float *R, int64_t r0, int64_t r1, const float *S, int64_t nS, int32_t d,
                            int32_t metric, double *out)
{
    for (int64_t i = r0; i < r1; ++i)
        for (int64_t j = 0; j < nS; ++j) {
            const float *q = R + i * (int64_t)d, *x = S + j * (int64_t)d;
            out[(i - r0) * nS + j] = (metric == 1) ? oracle_l1dist(q, x, d) : oracle_chi2dist(q, x, d);
        }
}

/*
 * Colour-histogram transformer (Sec. 4.1). frames is [nF][H][W][3] 8-bit RGB;
 * box i is boxes[5i..5i+4] = {frame, x0, y0, x1, y1}, the half-open pixel
 * rectangle [x0, x1) x [y0, y1). out is [nb][br*bg*bb]. Returns 0, or the
 * 1-based index of the first invalid box (out of the frame, empty, or more
 * than 2^24 pixels, where the count would not convert to FP32 exactly).
 */
int64_t oracle_color_hist(const uint8_t *frames, int64_t nF, int32_t H, int32_t W, const int32_t *boxes,
                          int64_t nb, int32_t br, int32_t bg, int32_t bb, float *out)
{
    const int32_t d = br * bg * bb;
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)d);
    if (!cnt) return -1;
    for (int64_t i = 0; i < nb; ++i) {
        const int32_t *bx = boxes + 5 * i;
        const int64_t f = bx[0];
        const int32_t x0 = bx[1], y0 = bx[2], x1 = bx[3], y1 = bx[4];
        if (f < 0 || f >= nF || x0 < 0 || y0 < 0 || x1 > W || y1 > H || x0 >= x1 || y0 >= y1 ||
            (int64_t)(x1 - x0) * (y1 - y0) > (1 << 24)) {
            free(cnt);
            return i + 1;
        }
        for (int32_t k = 0; k < d; ++k) cnt[k] = 0;
        for (int32_t y = y0; y < y1; ++y)
            for (int32_t x = x0; x < x1; ++x) {
                const uint8_t *px = frames + ((f * H + y) * (int64_t)W + x) * 3;
                const int32_t r = (px[0] * br) >> 8, g = (px[1] * bg) >> 8, b = (px[2] * bb) >> 8;
                cnt[(r * bg + g) * bb + b] += 1;
            }
        const float area = (float)((int64_t)(x1 - x0) * (y1 - y0));
        for (int32_t k = 0; k < d; ++k) out[i * d + k] = (float)cnt[k] / area;
    }
    free(cnt);
    return 0;
}

/*
 * Connected components of the graph on rows 0..n-1 with edges (a[e], b[e]):
 * label[i] = the smallest row index of i's component. Plain label propagation:
 * every row starts with its own index, each pass gives both ends of every edge
 * the smaller of their labels, until a pass changes nothing. Returns the
 * number of components, or -1 if an edge names a row outside [0, n).
 */
int64_t oracle_components(int64_t n, const int64_t *a, const int64_t *b, int64_t m, int64_t *label)
{
    for (int64_t e = 0; e < m; ++e)
        if (a[e] < 0 || a[e] >= n || b[e] < 0 || b[e] >= n) return -1;
    for (int64_t i = 0; i < n; ++i) label[i] = i;
    int changed = 1;
    while (changed) {
        changed = 0;
        for (int64_t e = 0; e < m; ++e) {
            const int64_t la = label[a[e]], lb = label[b[e]];
            const int64_t lo = (la < lb) ? la : lb;
            if (label[a[e]] != lo) {
                label[a[e]] = lo;
                changed = 1;
            }
            if (label[b[e]] != lo) {
                label[b[e]] = lo;
                changed = 1;
            }
        }
    }
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i) c += (label[i] == i);
    return c;
}

/*
 * Top-k with a histogram distance (metric 1 = L1, 2 = chi-square): for every query row,
 * the store rows ordered by (canonical distance, store row index), first min(k, nS) kept;
 * entries past that are -1 / -1.0. Returns 0, or -1 when the scratch allocation fails.
 */
int32_t oracle_hist_topk(const float *Q, int64_t nQ, const float *S, int64_t nS, int32_t d, int32_t metric,
                         int32_t k, int64_t *out_idx, double *out_d)
{
    oracle_cand *c = (oracle_cand *)malloc(sizeof(oracle_cand) * (size_t)(nS > 0 ? nS : 1));
    if (!c) return -1;
    const int64_t keep = (k < nS) ? k : nS;
    for (int64_t i = 0; i < nQ; ++i) {
        const float *q = Q + i * (int64_t)d;
        for (int64_t j = 0; j < nS; ++j) {
            const float *x = S + j * (int64_t)d;
            c[j].d2 = (metric == 1) ? oracle_l1dist(q, x, d) : oracle_chi2dist(q, x, d);
            c[j].j = j;
        }
        qsort(c, (size_t)nS, sizeof(oracle_cand), cand_cmp);
        for (int64_t t = 0; t < k; ++t) {
            out_idx[i * k + t] = (t < keep) ? c[t].j : -1;
            out_d[i * k + t] = (t < keep) ? c[t].d2 : -1.0;
        }
    }
    free(c);
    return 0;
}

/* Canonical dot product (k ascending, FP64, round to nearest; the products are exact). */
double oracle_dot(const float *q, const float *x, int32_t d)
{
    double s = 0.0;
    for (int32_t k = 0; k < d; ++k) s = s + (double)q[k] * (double)x[k];
    return s;
}

/* Inner-product threshold join: pairs with canonical q.x >= t; modes and output as oracle_join. */
int64_t oracle_ip_join(const float *R, int64_t nR, const float *S, int64_t nS, int32_t d, double t, int32_t mode,
                       int64_t *out_r, int64_t *out_s, int64_t cap)
{
    const float *T = (mode == 0) ? S : R;
    const int64_t nT = (mode == 0) ? nS : nR;
    int64_t cnt = 0;
    for (int64_t i = 0; i < nR; ++i) {
        int64_t j0 = (mode == 1) ? i + 1 : 0;
        for (int64_t j = j0; j < nT; ++j) {
            if (oracle_dot(R + i * (int64_t)d, T + j * (int64_t)d, d) >= t) {
                if (cnt < cap) {
                    out_r[cnt] = i;
                    out_s[cnt] = j;
                }
                ++cnt;
            }
        }
    }
    return cnt;
}
