// cc.cu -- q4 deduplication (Sec. 6.2 q4, Sec. 7.4.3): connected components of the
// epsilon self-join's pairs, and the two plan orders of Table 1.
//
// Components are found by concurrent union-find over a parent array:
//   k_cc_init   parent[i] = i;
//   k_cc_hook   one edge per thread: find both roots (path halving), hook the larger
//               root under the smaller with one atomicCAS on the larger root's slot,
//               retry when another edge hooked it first. A root is always the
//               smallest row of its tree (only larger roots are hooked under smaller
//               ones, and every parent is smaller than its child), so paths strictly
//               decrease and every find ends;
//   k_cc_label  label[i] = root of i, i.e. the smallest row of its component --
//               the same canonical labelling as the plain label propagation that
//               defines the result.
// A failed CAS means another thread hooked that root, so retries are bounded by the
// number of successful hooks (at most n - 1); no thread ever waits on another.
#include "kernels.h"

namespace dl {

namespace {

__device__ __forceinline__ int ld_parent(const int *p, int i) { return *((volatile const int *)(p + i)); }

__device__ __forceinline__ int cc_find(int *parent, int x)
{
    for (;;) {
        const int p = ld_parent(parent, x);
        if (p == x) return x;
        const int gp = ld_parent(parent, p);
        if (gp == p) return p;
        parent[x] = gp;   // path halving: gp is an ancestor of x, so any interleaving keeps a valid tree
        x = gp;
    }
}

__global__ void __launch_bounds__(256) k_cc_init(int *parent, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) parent[i] = i;
}

__global__ void __launch_bounds__(256)
    k_cc_hook(int *parent, int n, const int64_t *__restrict__ a, const int64_t *__restrict__ b, int64_t m, int *bad)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ua = __ldg(a + e), ub = __ldg(b + e);
        if (ua < 0 || ua >= n || ub < 0 || ub >= n) {
            atomicOr(bad, 1);
            continue;
        }
        int u = (int)ua, v = (int)ub;
        for (int tries = 0;; ++tries) {
            if (tries == (1 << 26)) {   // cannot happen (each failed CAS is another edge's hook); defensive
                atomicOr(bad, 2);
                break;
            }
            u = cc_find(parent, u);
            v = cc_find(parent, v);
            if (u == v) break;
            if (u > v) {
                const int t = u;
                u = v;
                v = t;
            }
            if (atomicCAS(parent + v, v, u) == v) break;   // v was still a root: hooked under u
        }
    }
}

// label[i] = smallest row of i's component; counts the roots (rows with label i), or with
// `keep` only the rows where keep[i] == target (those of other labels get -1).
__global__ void __launch_bounds__(256)
    k_cc_label(int *parent, int n, int64_t *label, const int32_t *__restrict__ keep, int32_t target,
               unsigned long long *n_roots)
{
    unsigned cnt = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int r = cc_find(parent, i);
        const bool kept = !keep || __ldg(keep + i) == target;
        label[i] = kept ? (int64_t)r : -1;
        cnt += (kept && r == i) ? 1u : 0u;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(n_roots, (unsigned long long)cnt);
}

// Match-then-filter: mark the components that hold at least one row labelled `target`.
__global__ void __launch_bounds__(256)
    k_cc_mark(const int64_t *__restrict__ label, int n, const int32_t *__restrict__ lab, int32_t target,
              unsigned *mark)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (__ldg(lab + i) == target) mark[label[i]] = 1u;
}

__global__ void __launch_bounds__(256) k_cc_count_marks(const unsigned *__restrict__ mark, int n,
                                                       unsigned long long *cnt_out)
{
    unsigned cnt = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) cnt += mark[i];
#pragma unroll
    for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(cnt_out, (unsigned long long)cnt);
}

// Store row i -> its caller row index (the ids a dedup join writes).
__global__ void __launch_bounds__(256) k_orig_ids(const int32_t *__restrict__ orig, int64_t n, int64_t *out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = orig[i];
}

// Filter-then-match: compact the store rows whose caller row is labelled `target`.
__global__ void __launch_bounds__(256)
    k_select_rows(const float *__restrict__ x32, const int32_t *__restrict__ orig, int64_t n, int d,
                  const int32_t *__restrict__ lab, int32_t target, float *xs, int64_t *ids_s,
                  unsigned long long *cnt)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w; i < n; i += nw) {
        const int32_t o = orig[i];
        if (__ldg(lab + o) != target) continue;   // warp-uniform
        unsigned long long pos = 0;
        if (lane == 0) pos = atomicAdd(cnt, 1ull);
        pos = __shfl_sync(0xffffffffu, pos, 0);
        for (int k = lane; k < d; k += 32) xs[pos * d + k] = x32[i * d + k];
        if (lane == 0) ids_s[pos] = o;
    }
}

int grid_for(int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)device_sm_count() * 8));
}

// Components of the graph with the given device edge lists; label (device, [n]) and the count.
int components_impl(int64_t n, const int64_t *a, const int64_t *b, int64_t m, int64_t *label,
                    const int32_t *keep, int32_t target, int64_t *n_comp, cudaStream_t st)
{
    if (n < 0 || m < 0 || n > 0x7fffffffLL) {
        set_error("components: n must be in [0, 2^31 - 1] and m >= 0");
        return DL_EINVAL;
    }
    if ((m > 0 && (!a || !b)) || (n > 0 && !label)) {
        set_error("components: NULL array");
        return DL_EINVAL;
    }
    if (n == 0) {
        if (n_comp) *n_comp = 0;
        return m > 0 ? (set_error("components: edges on an empty graph"), DL_EINVAL) : DL_OK;
    }
    void *blk = nullptr;
    int rc = dev_alloc(&blk, 256 + (size_t)n * 4, st);
    if (rc) return rc;
    unsigned long long *cnt = (unsigned long long *)blk;   // [0] roots [1] bad edge
    int *parent = (int *)((char *)blk + 256);
    cudaError_t e = cudaMemsetAsync(cnt, 0, 16, st);
    if (e == cudaSuccess) {
        k_cc_init<<<grid_for(n), 256, 0, st>>>(parent, (int)n);
        if (m > 0) k_cc_hook<<<grid_for(m), 256, 0, st>>>(parent, (int)n, a, b, m, (int *)(cnt + 1));
        k_cc_label<<<grid_for(n), 256, 0, st>>>(parent, (int)n, label, keep, target, cnt);
        count_launch(m > 0 ? 3 : 2);
        e = cudaGetLastError();
    }
    unsigned long long h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, cnt, 16, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(blk, st);
    if (e != cudaSuccess) return cuda_fail(e, "components");
    if (h[1] & 1) {
        set_error("components: an edge names a row outside [0, n)");
        return DL_EINVAL;
    }
    if (h[1] & 2) {
        set_error("components: union-find retry limit reached");
        return DL_ECUDA;
    }
    if (n_comp) *n_comp = (int64_t)h[0];
    return DL_OK;
}

int count_marked_components(const int64_t *label, int64_t n, const int32_t *lab, int32_t target, int64_t *out,
                            cudaStream_t st)
{
    void *blk = nullptr;
    int rc = dev_alloc(&blk, 256 + (size_t)n * 4, st);
    if (rc) return rc;
    unsigned long long *cnt = (unsigned long long *)blk;
    unsigned *mark = (unsigned *)((char *)blk + 256);
    cudaError_t e = cudaMemsetAsync(blk, 0, 256 + (size_t)n * 4, st);
    if (e == cudaSuccess) {
        k_cc_mark<<<grid_for(n), 256, 0, st>>>(label, (int)n, lab, target, mark);
        k_cc_count_marks<<<grid_for(n), 256, 0, st>>>(mark, (int)n, cnt);
        count_launch(2);
        e = cudaGetLastError();
    }
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, cnt, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(blk, st);
    if (e != cudaSuccess) return cuda_fail(e, "count_marked_components");
    *out = (int64_t)h;
    return DL_OK;
}

}  // namespace

}  // namespace dl

using namespace dl;

extern "C" {

int dl_components(int64_t n, const int64_t *pair_a, const int64_t *pair_b, int64_t m, int64_t *label,
                  int64_t *n_components, void *cuda_stream)
{
    dl::NvtxScope nvtx_scope("dl_components");
    clear_error();
    return components_impl(n, pair_a, pair_b, m, label, nullptr, 0, n_components, (cudaStream_t)cuda_stream);
}

int dl_dedup(const dl_store *X, int32_t metric, double eps, const int32_t *labels, int32_t target, int32_t plan,
             const dl_join_opts *opts, int64_t *comp, int64_t *n_distinct)
{
    dl::NvtxScope nvtx_scope("dl_dedup");
    clear_error();
    if (!X || !comp || !n_distinct) {
        set_error("dl_dedup: NULL argument");
        return DL_EINVAL;
    }
    if (plan != DL_DEDUP_ALL && plan != DL_DEDUP_FILTER_MATCH && plan != DL_DEDUP_MATCH_FILTER) {
        set_error("dl_dedup: bad plan %d", plan);
        return DL_EINVAL;
    }
    if (plan != DL_DEDUP_ALL && !labels) {
        set_error("dl_dedup: the label plans need labels");
        return DL_EINVAL;
    }
    dl_join_opts o;
    if (opts)
        o = *opts;
    else
        dl_join_opts_default(&o);
    o.self_mode = DL_SELF_UPPER;
    o.out_capacity = 0;
    cudaStream_t st = (cudaStream_t)o.cuda_stream;
    const int64_t n = X->n;
    const int d = X->d;
    int rc = DL_OK;
    dl_result *res = nullptr;
    if (plan == DL_DEDUP_FILTER_MATCH) {
        // the rows labelled `target`, as a store of their own whose ids are their caller rows
        void *blk = nullptr;
        const size_t bx = ((size_t)std::max<int64_t>(n, 1) * d * 4 + 255) & ~size_t(255);
        rc = dev_alloc(&blk, 256 + bx + (size_t)std::max<int64_t>(n, 1) * 8, st);
        if (rc) return rc;
        unsigned long long *cnt = (unsigned long long *)blk;
        float *xs = (float *)((char *)blk + 256);
        int64_t *ids_s = (int64_t *)((char *)blk + 256 + bx);
        cudaError_t e = cudaMemsetAsync(cnt, 0, 8, st);
        if (e == cudaSuccess && n > 0) {
            k_select_rows<<<grid_for(n * 32), 256, 0, st>>>(X->x32, X->orig, n, d, labels, target, xs, ids_s, cnt);
            count_launch();
            e = cudaGetLastError();
        }
        unsigned long long ns = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&ns, cnt, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            dev_free(blk, st);
            return cuda_fail(e, "dl_dedup select");
        }
        dl_store *sub = nullptr;
        if (ns > 0) {
            rc = store_create_impl(&sub, ids_s, xs, (int64_t)ns, d, DL_MEM_DEVICE, st, nullptr);
            if (!rc) sub->unit = X->unit;
            if (!rc) rc = sim_join_impl(sub, nullptr, metric, eps, &o, &res, nullptr);
        }
        if (!rc) {
            const int64_t m = res ? res->count : 0;
            rc = components_impl(n, m ? res->d_r : nullptr, m ? res->d_s : nullptr, m, comp, labels, target,
                                 n_distinct, st);
        }
        if (res) dl_result_free(res);
        if (sub) dl_store_destroy(sub);
        dev_free(blk, st);
        return rc;
    }
    // every row: the self-join writes caller rows, then components over all rows
    void *blk = nullptr;
    rc = dev_alloc(&blk, (size_t)std::max<int64_t>(n, 1) * 8, st);
    if (rc) return rc;
    int64_t *rows = (int64_t *)blk;
    if (n > 0) {
        k_orig_ids<<<grid_for(n), 256, 0, st>>>(X->orig, n, rows);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            dev_free(blk, st);
            return cuda_fail(e, "k_orig_ids launch");
        }
    }
    rc = sim_join_impl(X, nullptr, metric, eps, &o, &res, rows);
    if (!rc) {
        const int64_t m = res->count;
        rc = components_impl(n, m ? res->d_r : nullptr, m ? res->d_s : nullptr, m, comp, nullptr, 0, n_distinct, st);
    }
    if (res) dl_result_free(res);
    dev_free(blk, st);
    if (!rc && plan == DL_DEDUP_MATCH_FILTER && n > 0) rc = count_marked_components(comp, n, labels, target, n_distinct, st);
    return rc;
}

}  // extern "C"
