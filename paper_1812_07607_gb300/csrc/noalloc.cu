// noalloc.cu -- an exact epsilon-join entry point that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they need a
// join: code running while a memory planner owns the whole device, real-time
// loops that must not hit the allocator, or hosts that forbid cudaMalloc after
// start-up. dl_sim_join_noalloc serves them: the caller passes its own device
// buffers for the inputs (features, ids) and the outputs (id pairs), and the
// only working memory the join needs -- four counters and the list of pairs
// whose FP32 distance lies within its error bound of eps^2 -- lives in the
// file-scope device array below, which every GPU that loads this library holds
// until the process exits.
//
// It runs the exact FP32 path (K8 in exact mode, then the K6 recheck), so its
// result is the same set dl_sim_join returns. The rows come straight from the
// caller, so the domain dl_store_create enforces (every feature finite, |x| <=
// 2^40, which the FP32 and FP64 error bounds assume) is checked here by a small
// kernel that raises a flag in the scratch counters.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "kernels.h"

namespace dl {

// At most this many pairs may fall inside the FP32 error band in one call
// (8 bytes each); a call that needs more is rejected with DL_EOVERFLOW.
constexpr unsigned long long kNoAllocBandMax = 65536;
constexpr size_t kNoAllocCounterBytes = 256;
constexpr size_t kNoAllocScratchBytes = kNoAllocCounterBytes + kNoAllocBandMax * sizeof(uint2);   // 512 KiB + 256 B

// Counters ([0] pairs out, [1] band pairs, [2] FP64 evaluations, [3] domain flag) followed
// by the band list.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Raises *flag when any of the n*d features of X is non-finite or above 2^40 in
// magnitude (the domain of the error bounds; dl_store_create rejects the same).
__global__ void __launch_bounds__(256) k_noalloc_domain(const float *__restrict__ X, int64_t count,
                                                        unsigned long long *flag)
{
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        if (!(fabsf(__ldg(X + i)) <= 1099511627776.0f)) bad = true;   // also catches NaN
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1ull);
}

static int launch_domain(const float *X, int64_t count, unsigned long long *flag, cudaStream_t st)
{
    if (count <= 0) return DL_OK;
    const int64_t want = (count + 255) / 256;
    const int grid = (int)(want < (int64_t)device_sm_count() * 8 ? want : (int64_t)device_sm_count() * 8);
    k_noalloc_domain<<<grid, 256, 0, st>>>(X, count, flag);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_noalloc_domain launch");
    return DL_OK;
}

static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[64];   // device address of g_noalloc_scratch, per device

// Host code cannot use the array's name as a device address; look the address
// up once per device (with that device current) and reuse it.
static int noalloc_scratch(void **out)
{
    int dev = 0;
    DL_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("dl_sim_join_noalloc: device index %d out of range", dev);
        return DL_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return DL_OK;
}

}  // namespace dl

using namespace dl;

extern "C" int dl_sim_join_noalloc(const float *R, const int64_t *r_ids, int64_t nR, const float *S,
                                   const int64_t *s_ids, int64_t nS, int32_t d, double eps, int32_t self_mode,
                                   int64_t *out_r, int64_t *out_s, int64_t out_cap, int64_t *n_out,
                                   void *cuda_stream)
{
    dl::NvtxScope nvtx_scope("dl_sim_join_noalloc");
    clear_error();
    if (!n_out) {
        set_error("dl_sim_join_noalloc: n_out is NULL");
        return DL_EINVAL;
    }
    *n_out = 0;
    const bool self = (S == nullptr);
    if (self) {
        s_ids = r_ids;
        nS = nR;
    }
    if (d < 1 || d > 1024) {
        set_error("dl_sim_join_noalloc: d=%d out of range [1, 1024]", d);
        return DL_EINVAL;
    }
    if (nR < 0 || nS < 0 || nR >= (int64_t(1) << 31) || nS >= (int64_t(1) << 31)) {
        set_error("dl_sim_join_noalloc: row counts must be in [0, 2^31)");
        return DL_EINVAL;
    }
    if ((nR > 0 && (!R || !r_ids)) || (!self && nS > 0 && !s_ids)) {
        set_error("dl_sim_join_noalloc: NULL input pointer");
        return DL_EINVAL;
    }
    if (std::isnan(eps) || eps < 0.0) {
        set_error("dl_sim_join_noalloc: eps must be >= 0 (got %g)", eps);
        return DL_EINVAL;
    }
    if (self_mode != DL_SELF_UPPER && self_mode != DL_SELF_FULL) {
        set_error("dl_sim_join_noalloc: bad self_mode %d", self_mode);
        return DL_EINVAL;
    }
    if (out_cap < 0 || (out_cap > 0 && (!out_r || !out_s))) {
        set_error("dl_sim_join_noalloc: bad output buffers");
        return DL_EINVAL;
    }
    // The recheck reads rows as 16-byte vectors when d % 4 == 0, and ids and pairs are
    // 8-byte words: refuse pointers those accesses would fault on, before any launch.
    const uintptr_t row_align = (d % 4 == 0) ? 15u : 3u;
    if ((((uintptr_t)R | (uintptr_t)S) & row_align) != 0) {
        set_error("dl_sim_join_noalloc: R and S must be %d-byte aligned for d=%d", (int)row_align + 1, d);
        return DL_EINVAL;
    }
    if ((((uintptr_t)r_ids | (uintptr_t)s_ids | (uintptr_t)out_r | (uintptr_t)out_s) & 7u) != 0) {
        set_error("dl_sim_join_noalloc: ids and output pairs must be 8-byte aligned");
        return DL_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    void *scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    unsigned long long *cnt = (unsigned long long *)scratch;
    uint2 *band = (uint2 *)((char *)scratch + kNoAllocCounterBytes);

    // every call starts from zeroed counters (the array keeps the previous call's contents)
    DL_CUDA_TRY(cudaMemsetAsync(cnt, 0, kNoAllocCounterBytes, st));
    rc = launch_domain(R, nR * (int64_t)d, cnt + 3, st);
    if (!rc && !self) rc = launch_domain(S, nS * (int64_t)d, cnt + 3, st);
    if (rc) return rc;

    const double e2 = eps * eps;
    const double g64 = gamma64(d), g32 = gamma32(d);
    const double abs32 = (double)(d + 8) * 1.401298464324817e-45 * 2.0;
    const float t_acc = f32_rd(e2 * (1.0 - g64) * (1.0 - g32) * (1.0 - 8.881784197001252e-16) - abs32);
    const float t_rej = f32_ru(e2 * (1.0 + 2.0 * g64) * (1.0 + g32) * (1.0 + 8.881784197001252e-16) + abs32);
    const bool mirror = self && self_mode == DL_SELF_FULL;

    JoinOut jo{};
    jo.r_ids = r_ids;
    jo.s_ids = s_ids;
    jo.out_r = out_r;
    jo.out_s = out_s;
    jo.out_cnt = cnt + 0;
    jo.out_cap = (unsigned long long)out_cap;
    jo.band = band;
    jo.band_cnt = cnt + 1;
    jo.band_cap = kNoAllocBandMax;
    jo.mirror = mirror ? 1 : 0;
    jo.orig = nullptr;   // caller's row order is the store order here

    if (nR > 0 && nS > 0) {
        SimtParams sp{};
        sp.R = R;
        sp.S = self ? R : S;
        sp.nR = (int)nR;
        sp.nS = (int)nS;
        sp.d = d;
        sp.upper = self ? 1 : 0;
        sp.tiles_m = 0;
        sp.exact = 1;
        sp.metric = 0;   // squared L2
        sp.t_acc = t_acc;
        sp.t_rej = t_rej;
        sp.out = jo;
        rc = launch_simt_join(sp, st);
        if (rc) return rc;
        rc = launch_recheck(band, cnt + 1, kNoAllocBandMax, R, self ? R : S, d, e2, t_acc, t_rej, jo, cnt + 2,
                            device_sm_count() * 8, st);
        if (rc) return rc;
    }
    if (mirror) {
        rc = launch_diag(r_ids, nR, out_r, out_s, cnt + 0, (unsigned long long)out_cap, st);
        if (rc) return rc;
    }
    unsigned long long h[4] = {0, 0, 0, 0};
    DL_CUDA_TRY(cudaMemcpyAsync(h, cnt, sizeof h, cudaMemcpyDeviceToHost, st));
    DL_CUDA_TRY(cudaStreamSynchronize(st));
    if (h[3]) {
        set_error("dl_sim_join_noalloc: a feature is non-finite or exceeds 2^40 in magnitude; the output is "
                  "unspecified");
        return DL_EINVAL;
    }
    *n_out = (int64_t)h[0];
    if (h[1] > kNoAllocBandMax) {
        set_error("dl_sim_join_noalloc: %llu pairs fell inside the FP32 error band, more than the %llu the "
                  "static scratch holds; the output is incomplete (use dl_sim_join)",
                  h[1], kNoAllocBandMax);
        return DL_EOVERFLOW;
    }
    if (h[0] > (unsigned long long)out_cap) {
        set_error("dl_sim_join_noalloc: %llu pairs exceed out_cap %lld", h[0], (long long)out_cap);
        return DL_EOVERFLOW;
    }
    return DL_OK;
}
