// hist.cu -- the colour-histogram transformer (Sec. 4.1 "Transformers": colour
// histogram features for image matching), feeding the join's stores directly.
//
// A patch is a box {frame, x0, y0, x1, y1} (half-open) of a frame of 8-bit
// interleaved RGB pixels. Channel value v falls in bin floor(v*b/256) of its
// channel's b bins; the joint bin is (r*bg + g)*bb + b; the histogram is
// count / (pixels of the box), one correctly rounded FP32 division per bin, so
// the output is bit-exact.
//
// The work is HBM-bound (three bytes per pixel in, 4 d bytes per box out):
//   k_hist_plan   one CTA: validates every box and cuts it into items of at
//                 most kItemSegs 48-byte segments (prefix sum of item counts),
//                 and writes the item -> (box, index in box) table;
//   k_hist_count  persistent CTAs take items from an atomic counter (the next
//                 item is fetched while the current one is counted). A lane
//                 owns one 48-byte segment of one box row: three aligned 16-byte
//                 loads plus the next 4-byte word (a pixel may straddle the
//                 segment's end). Every segment starts at the same byte phase
//                 (48 is a multiple of 3), so the 16 pixel positions inside it
//                 are compile-time offsets of one of three phases. Each pixel
//                 adds 1 to its bin in its lane's copy of the CTA's shared
//                 histogram (up to 32 interleaved copies, so that the lanes of
//                 a warp never share a bank); power-of-two bin counts take a
//                 mask, one multiply and a shift. Each item ends with one
//                 global atomic per non-zero bin, and the last item of a box
//                 to finish writes its histogram, counts / area.
#include "kernels.h"

namespace dl {

namespace {

constexpr int kHistThreads = 128;
constexpr int kItemSegs = 1024;     // segments (16 pixels each) per work item
constexpr int kPlanThreads = 1024;
constexpr int kMaxSmemHist = 32768; // bytes of interleaved shared histogram copies per CTA

struct HistParams {
    const uint8_t *frames;
    int64_t frame_bytes_total;      // n_frames * H * W * 3
    int64_t n_frames;
    int32_t H, W;
    const int32_t *boxes;
    int64_t nb;
    int32_t br, bg, bb, d;
    uint32_t gM, gK, gS;            // gather form of the bin (see BinSpec), when gather != 0
    int32_t gather;
    int64_t *item_off;              // [nb + 1] first item of each box (prefix sum)
    int2 *item_box;                 // [table_cap] {box, item index within the box} of each item
    int64_t table_cap;              // items past this are located by binary search instead
    unsigned *counts;               // [nb][d]
    unsigned long long *next_item;  // work counter
    int *bad;                       // set to 1 + box index of an invalid box
    int *box_done;                  // [nb] items of the box counted so far
    int lcopies;                    // log2 of the shared histogram copies (>= 2)
    float *out;
};

__device__ __forceinline__ int64_t box_segs_per_row(int32_t w) { return (3 * (int64_t)w + 15 + 47) / 48; }

// One CTA: item counts of every box, their exclusive prefix sum, and the validity check.
__global__ void __launch_bounds__(kPlanThreads) k_hist_plan(HistParams p)
{
    __shared__ int64_t warp_tot[kPlanThreads / 32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t b0 = 0; b0 < p.nb; b0 += kPlanThreads) {
        const int64_t b = b0 + threadIdx.x;
        int64_t items = 0;
        if (b < p.nb) {
            const int32_t *bx = p.boxes + 5 * b;
            const int32_t f = bx[0], x0 = bx[1], y0 = bx[2], x1 = bx[3], y1 = bx[4];
            const bool ok = f >= 0 && f < p.n_frames && x0 >= 0 && y0 >= 0 && x1 <= p.W && y1 <= p.H && x0 < x1 &&
                            y0 < y1 && (int64_t)(x1 - x0) * (y1 - y0) <= (1ll << 24);
            if (ok) {
                const int64_t segs = box_segs_per_row(x1 - x0) * (y1 - y0);
                items = (segs + kItemSegs - 1) / kItemSegs;
            } else {
                atomicCAS(p.bad, 0, (int)(b + 1 < 0x7fffffff ? b + 1 : 0x7fffffff));
            }
        }
        // block-wide inclusive scan of items
        int64_t v = items;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) warp_tot[wid] = v;
        __syncthreads();
        if (wid == 0) {
            int64_t t = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t u = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += u;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        const int64_t incl = v + (wid ? warp_tot[wid - 1] : 0) + carry;
        if (b < p.nb) {
            p.item_off[b] = incl - items;
            for (int64_t t = 0; t < items && incl - items + t < p.table_cap; ++t)
                p.item_box[incl - items + t] = make_int2((int)b, (int)t);
        }
        __syncthreads();
        if (threadIdx.x == kPlanThreads - 1) carry = incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        p.item_off[p.nb] = carry;
        *p.next_item = 0ull;
    }
}

struct BinSpec {
    int br, bg, bb, gbb;    // bins per channel, gbb = bg * bb
    // gather form (power-of-two bins whose fields do not collide; checked on the host):
    // bin = ((v & M) * K mod 2^32) >> S for the packed pixel v = r | g << 8 | b << 16
    uint32_t M, K, S;
};

// *addr += v in shared memory when p holds (a predicated reduction, no branch).
__device__ __forceinline__ void red_shared_if(unsigned *addr, unsigned v, bool p)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(addr);
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q red.shared.add.u32 [%0], %1;\n\t}" ::"r"(a), "r"(v),
        "r"((unsigned)p)
        : "memory");
}

template <bool GATHER>
__device__ __forceinline__ int pixel_bin(uint32_t v, const BinSpec &b)
{
    if constexpr (GATHER) {
        return (int)(((v & b.M) * b.K) >> b.S);
    } else {
        const int r = (int)(v & 255u), g = (int)__byte_perm(v, 0u, 0x4441), c = (int)__byte_perm(v, 0u, 0x4442);
        return ((r * b.br) >> 8) * b.gbb + ((g * b.bg) >> 8) * b.bb + ((c * b.bb) >> 8);
    }
}

// Direct form: every valid pixel adds 1 to its bin in this lane's copy of the histogram
// (2^lc interleaved copies, copy = lane mod 2^lc, word = bin * 2^lc + copy). With 32 copies
// every lane of a warp owns one bank, so a warp's reductions never conflict, whatever bins
// its pixels fall in.
template <int PHI, bool GATHER>
__device__ __forceinline__ void seg_count_direct(const uint32_t (&w)[13], uint32_t valid, const BinSpec &b,
                                                 unsigned *sh_lane, int lc)
{
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int o = PHI + 3 * i;
        const int wi = o >> 2, sft = (o & 3) * 8;
        const uint32_t v = sft ? __funnelshift_r(w[wi], w[wi + 1], sft) : w[wi];
        red_shared_if(sh_lane + (pixel_bin<GATHER>(v, b) << lc), 1u, (valid >> i) & 1u);
    }
}

template <bool GATHER>
__device__ __forceinline__ void seg_count_phase(int phi, const uint32_t (&w)[13], uint32_t valid, const BinSpec &b,
                                                unsigned *sh, int lc)
{
    if (phi == 0) seg_count_direct<0, GATHER>(w, valid, b, sh, lc);
    else if (phi == 1) seg_count_direct<1, GATHER>(w, valid, b, sh, lc);
    else seg_count_direct<2, GATHER>(w, valid, b, sh, lc);
}

__device__ __forceinline__ uint32_t byte_at(const uint8_t *base, int64_t a, int64_t lo, int64_t hi)
{
    return (a >= lo && a < hi) ? (uint32_t)base[a] : 0u;
}

template <bool GATHER>
__global__ void __launch_bounds__(kHistThreads, 8) k_hist_count(HistParams p)
{
    extern __shared__ __align__(16) unsigned sh_hist[];   // [d][2^lcopies]
    __shared__ long long s_item[2];          // this item and the next one (fetched while this one runs)
    __shared__ bool s_last;
    BinSpec bs;
    bs.br = p.br, bs.bg = p.bg, bs.bb = p.bb, bs.gbb = p.bg * p.bb;
    bs.M = p.gM, bs.K = p.gK, bs.S = p.gS;
    const int lc = p.lcopies;
    const int64_t total_items = p.item_off[p.nb];
    if (threadIdx.x == 0) s_item[0] = (long long)atomicAdd(p.next_item, 1ull);
    for (int k = threadIdx.x; k < (p.d << lc) / 4; k += kHistThreads)
        reinterpret_cast<uint4 *>(sh_hist)[k] = make_uint4(0u, 0u, 0u, 0u);
    for (int it = 0;; ++it) {
        __syncthreads();
        const int64_t item = s_item[it & 1];
        if (item >= total_items) break;
        if (threadIdx.x == 0) s_item[(it + 1) & 1] = (long long)atomicAdd(p.next_item, 1ull);
        int64_t box, local;
        if (item < p.table_cap) {
            const int2 e = p.item_box[item];
            box = e.x;
            local = e.y;
        } else {
            // the box holding this item: last b with item_off[b] <= item
            int64_t lo = 0, hi = p.nb - 1;
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (p.item_off[mid] <= item) lo = mid;
                else hi = mid - 1;
            }
            box = lo;
            local = item - p.item_off[box];
        }
        const int32_t *bx = p.boxes + 5 * box;
        const int64_t f = bx[0];
        const int32_t x0 = bx[1], y0 = bx[2], x1 = bx[3], y1 = bx[4];
        const uint32_t wbytes = 3u * (uint32_t)(x1 - x0);                       // bytes of one box row
        const uint32_t spr = (uint32_t)box_segs_per_row(x1 - x0);
        const uint32_t seg_total = spr * (uint32_t)(y1 - y0);     // < 2^26: boxes hold at most 2^24 pixels
        const uint32_t sg0 = (uint32_t)local * kItemSegs;
        // row = umulhi(sg, spr_inv) is exact or one too high for spr >= 2 (spr_inv >= 2^32 / spr, and
        // sg < 2^26 keeps the excess below 1/64); spr == 1 is the identity
        const uint32_t spr_inv = spr > 1 ? 0xffffffffu / spr + 1u : 0u;
        const uint32_t sg1 = min(sg0 + kItemSegs, seg_total);
        const int64_t base = ((f * p.H + y0) * p.W + x0) * 3;                   // first byte of the box
        const int64_t pitch = 3 * (int64_t)p.W;
        for (uint32_t sg = sg0 + threadIdx.x; sg < sg1; sg += kHistThreads) {
            uint32_t row = spr > 1 ? __umulhi(sg, spr_inv) : sg;
            if (row * spr > sg) --row;
            const uint32_t j = sg - row * spr;
            const int64_t s = base + row * pitch;                              // first byte of the box row
            const uint32_t lead = (uint32_t)s & 15u;                            // s - s0
            const int64_t a = s - lead + 48 * (int64_t)j;                      // this segment
            // byte offsets (from the row start) of the segment's window: [48 j - lead, 48 j - lead + 48)
            const int32_t off = 48 * (int32_t)j - (int32_t)lead;
            if (off >= (int32_t)wbytes) continue;
            const int phi = (int)(lead % 3u);
            // pixel i of the segment starts at row byte off + phi + 3 i; keep 0 <= that < wbytes
            const int32_t first = off + phi;
            const int32_t i_lo = first >= 0 ? 0 : (-first) / 3;
            const int32_t n_in = ((int32_t)wbytes - first) / 3;
            const int32_t i_hi = n_in < 16 ? n_in : 16;
            const uint32_t valid = (0xffffu >> (16 - i_hi)) & ~((1u << i_lo) - 1u);
            uint32_t w[13];
            if (a + 64 <= p.frame_bytes_total) {
                const uint4 *q = reinterpret_cast<const uint4 *>(p.frames + a);
                const uint4 v0 = __ldg(q), v1 = __ldg(q + 1), v2 = __ldg(q + 2);
                w[0] = v0.x, w[1] = v0.y, w[2] = v0.z, w[3] = v0.w;
                w[4] = v1.x, w[5] = v1.y, w[6] = v1.z, w[7] = v1.w;
                w[8] = v2.x, w[9] = v2.y, w[10] = v2.z, w[11] = v2.w;
                w[12] = __ldg(reinterpret_cast<const uint32_t *>(p.frames + a + 48));
            } else {
                // the end of the frame buffer: byte loads that stay inside the box row
                const int64_t e = s + wbytes;
#pragma unroll
                for (int k = 0; k < 13; ++k) {
                    const int64_t b = a + 4 * k;
                    w[k] = byte_at(p.frames, b, s, e) | (byte_at(p.frames, b + 1, s, e) << 8) |
                           (byte_at(p.frames, b + 2, s, e) << 16) | (byte_at(p.frames, b + 3, s, e) << 24);
                }
            }
            seg_count_phase<GATHER>(phi, w, valid, bs, sh_hist + (threadIdx.x & ((1 << lc) - 1)), lc);
        }
        __syncthreads();
        unsigned *gc = p.counts + box * p.d;
        for (int k = threadIdx.x; k < p.d; k += kHistThreads) {
            unsigned c = 0;
            for (int q0 = 0; q0 < (1 << lc); q0 += 4) {
                const int q = (q0 + 4 * k) & ((1 << lc) - 1);   // rotated start: neighbouring bins read other banks
                uint4 *cell = reinterpret_cast<uint4 *>(sh_hist + (k << lc) + q);
                const uint4 t = *cell;
                *cell = make_uint4(0u, 0u, 0u, 0u);   // leaves the copies zeroed for the next item
                c += t.x + t.y + t.z + t.w;
            }
            if (c) atomicAdd(gc + k, c);
        }
        // the box's last item to finish turns its counts into the histogram
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            const int n_items = (int)(p.item_off[box + 1] - p.item_off[box]);
            s_last = atomicAdd(p.box_done + box, 1) == n_items - 1;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            const float area = (float)((int64_t)(x1 - x0) * (y1 - y0));
            for (int k = threadIdx.x; k < p.d; k += kHistThreads)
                p.out[box * p.d + k] = __fdiv_rn((float)__ldcg(gc + k), area);
        }
    }
}

// Power-of-two bins: the top bits of each channel, masked out of the packed pixel, land in bin
// order at the top of the 32-bit word after one multiply by K = 2^t (1 + 2^(8+lg) + 2^(16+lr+lg))
// with t = 8 - lr - lg, so that a shift by 32 - log2(d) leaves the bin -- as long as no shifted
// copy of another field, and no carry, reaches those bits. Checked here on every one of the
// br*bg*bb field combinations; false means the multiply-and-shift form is used instead.
bool bin_gather_form(int br, int bg, int bb, uint32_t *M, uint32_t *K, uint32_t *S)
{
    auto lg2 = [](int x) { int l = 0; while ((1 << l) < x) ++l; return l; };
    if ((br & (br - 1)) || (bg & (bg - 1)) || (bb & (bb - 1))) return false;
    const int lr = lg2(br), lgg = lg2(bg), lb = lg2(bb), L = lr + lgg + lb;
    if (L == 0) {   // one bin
        *M = 0u, *K = 0u, *S = 0u;
        return true;
    }
    const int t = 8 - lr - lgg;
    if (t < 0) return false;
    const uint32_t m = ((uint32_t)(br - 1) << (8 - lr)) | ((uint32_t)(bg - 1) << (16 - lgg)) |
                       ((uint32_t)(bb - 1) << (24 - lb));
    const uint32_t k = (1u + (1u << (8 + lgg)) + (1u << (16 + lr + lgg))) << t;
    const uint32_t sh = (uint32_t)(32 - L);
    for (int r = 0; r < br; ++r)
        for (int g = 0; g < bg; ++g)
            for (int b = 0; b < bb; ++b) {
                const uint32_t v = ((uint32_t)r << (8 - lr)) | ((uint32_t)g << (16 - lgg)) | ((uint32_t)b << (24 - lb));
                if (((v * k) >> sh) != (uint32_t)((r * bg + g) * bb + b)) return false;
            }
    *M = m;
    *K = k;
    *S = sh;
    return true;
}

}  // namespace

int color_hist_impl(const uint8_t *frames, int64_t n_frames, int32_t H, int32_t W, const int32_t *boxes, int64_t nb,
                    int32_t br, int32_t bg, int32_t bb, float *out, float *count_ms, cudaStream_t st)
{
    if (nb < 0 || n_frames < 0 || H < 0 || W < 0) {
        set_error("dl_color_hist: negative size");
        return DL_EINVAL;
    }
    if (br < 1 || br > 256 || bg < 1 || bg > 256 || bb < 1 || bb > 256 || (int64_t)br * bg * bb > 1024) {
        set_error("dl_color_hist: bins must be in [1, 256] with br*bg*bb <= 1024");
        return DL_EINVAL;
    }
    if (nb == 0) return DL_OK;
    if (!frames || !boxes || !out || n_frames == 0 || H == 0 || W == 0) {
        set_error("dl_color_hist: null pointer or empty frames with boxes to read");
        return DL_EINVAL;
    }
    if ((reinterpret_cast<uintptr_t>(frames) & 15) != 0 || (reinterpret_cast<uintptr_t>(boxes) & 3) != 0) {
        set_error("dl_color_hist: frames must be 16-byte aligned and boxes 4-byte aligned");
        return DL_EINVAL;
    }
    const int d = br * bg * bb;
    HistParams p{};
    p.frames = frames;
    p.frame_bytes_total = n_frames * H * (int64_t)W * 3;
    p.n_frames = n_frames;
    p.H = H;
    p.W = W;
    p.boxes = boxes;
    p.nb = nb;
    p.br = br;
    p.bg = bg;
    p.bb = bb;
    p.d = d;
    p.gather = bin_gather_form(br, bg, bb, &p.gM, &p.gK, &p.gS) ? 1 : 0;
    p.out = out;
    // scratch: item offsets, counts, work counter, error word
    const size_t off_bytes = ((size_t)(nb + 1) * 8 + 255) & ~size_t(255);
    const size_t cnt_bytes = ((size_t)nb * d * 4 + 255) & ~size_t(255);   // keeps the 8-byte counter aligned
    // item table: every box has at most ceil(H * segments-per-frame-row / kItemSegs) items
    const int64_t max_items_box = (H * ((3 * (int64_t)W + 62) / 48) + kItemSegs - 1) / kItemSegs;
    p.table_cap = std::min<int64_t>(nb * max_items_box, (int64_t)1 << 22);
    const size_t tab_bytes = ((size_t)p.table_cap * 8 + 255) & ~size_t(255);
    const size_t done_bytes = ((size_t)nb * 4 + 255) & ~size_t(255);
    const size_t bytes = off_bytes + cnt_bytes + 256 + done_bytes + tab_bytes;
    void *blk = nullptr;
    int rc = dev_alloc(&blk, bytes, st);
    if (rc) return rc;
    p.item_off = reinterpret_cast<int64_t *>(blk);
    p.counts = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(blk) + off_bytes);
    p.next_item = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(blk) + off_bytes + cnt_bytes);
    p.bad = reinterpret_cast<int *>(p.next_item + 1);
    p.box_done = reinterpret_cast<int *>(reinterpret_cast<char *>(blk) + off_bytes + cnt_bytes + 256);
    p.item_box = reinterpret_cast<int2 *>(reinterpret_cast<char *>(blk) + off_bytes + cnt_bytes + 256 + done_bytes);
    static thread_local int *h_bad = nullptr;   // pinned error word of this host thread
    cudaError_t e = cudaSuccess;
    if (!h_bad) e = cudaMallocHost(&h_bad, sizeof(int));
    if (e != cudaSuccess) {
        h_bad = nullptr;
        dev_free(blk, st);
        return cuda_fail(e, "cudaMallocHost");
    }
    cudaEvent_t ev[2] = {nullptr, nullptr};
    e = cudaMemsetAsync(p.counts, 0, cnt_bytes + 256 + done_bytes, st);   // counts, counter, error word, box_done
    if (e == cudaSuccess) {
        k_hist_plan<<<1, kPlanThreads, 0, st>>>(p);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        int sms = device_sm_count();
        p.lcopies = 5;
        while (p.lcopies > 2 && ((size_t)d << p.lcopies) * 4 > (size_t)kMaxSmemHist) --p.lcopies;
        const size_t smem = ((size_t)d << p.lcopies) * 4;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hist_count<true>, kHistThreads, smem);
        if (e == cudaSuccess && count_ms) {
            e = cudaEventCreate(&ev[0]);
            if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
            if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
        }
        if (e == cudaSuccess) {
            if (p.gather) k_hist_count<true><<<sms * (per_sm > 0 ? per_sm : 1), kHistThreads, smem, st>>>(p);
            else k_hist_count<false><<<sms * (per_sm > 0 ? per_sm : 1), kHistThreads, smem, st>>>(p);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess && ev[1]) e = cudaEventRecord(ev[1], st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_bad, p.bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && ev[0]) e = cudaEventElapsedTime(count_ms, ev[0], ev[1]);
    for (auto &x : ev)
        if (x) cudaEventDestroy(x);
    count_launch(2);
    dev_free(blk, st);
    if (e != cudaSuccess) return cuda_fail(e, "dl_color_hist");
    const int bad = *h_bad;
    if (bad) {
        set_error("dl_color_hist: box %d is invalid (outside its frame, empty, or more than 2^24 pixels)", bad - 1);
        return DL_EINVAL;
    }
    return DL_OK;
}

}  // namespace dl

using namespace dl;

extern "C" int dl_color_hist(const uint8_t *frames, int64_t n_frames, int32_t H, int32_t W, const int32_t *boxes,
                             int64_t n_boxes, int32_t br, int32_t bg, int32_t bb, float *out, float *count_ms,
                             void *cuda_stream)
{
    dl::NvtxScope nvtx_scope("dl_color_hist");
    clear_error();
    if (count_ms) *count_ms = 0.f;
    return color_hist_impl(frames, n_frames, H, W, boxes, n_boxes, br, bg, bb, out, count_ms,
                           (cudaStream_t)cuda_stream);
}
