// exact.cuh -- the exact decision for one pair: an FP32 sum with its bound first, then a
// float-float sum with a much tighter bound, and the canonical FP64 sum only for the pairs
// neither can place (in practice, pairs whose distance ties eps^2 to about 1e-10).
#pragma once

#include <cstdint>

namespace dl {

// FP32 thresholds for a squared threshold e2 at dimension d: accept if the FP32
// distance sum D32 <= t_acc, reject if D32 > t_rej, else evaluate the canonical
// FP64 sum. Sound for |D32 - D| <= (d+8) 2^-24 D + (d+8) 2^-148 and for the
// canonical sum's (d+4) 2^-53 relative error; the (1 -/+ 2^-50) factors absorb the
// roundings of this very computation.
__device__ __forceinline__ void fp32_thresholds(double e2, int d, float *t_acc, float *t_rej)
{
    const double g64 = (double)(d + 4) * 1.1102230246251565e-16;
    const double g32 = (double)(d + 8) * 5.9604644775390625e-08;
    const double abs32 = (double)(d + 8) * 1.401298464324817e-45 * 2.0;
    *t_acc = __double2float_rd(e2 * (1.0 - g64) * (1.0 - g32) * (1.0 - 8.881784197001252e-16) - abs32);
    *t_rej = __double2float_ru(e2 * (1.0 + 2.0 * g64) * (1.0 + g32) * (1.0 + 8.881784197001252e-16) + abs32);
}

// ---- float-float stage. The FP32 bound leaves a relative zone of about 2 (d+8) 2^-24 around
// eps^2 undecided, and the canonical FP64 sum that settles it is a chain of d dependent
// additions at the FP64 rate. Between the two sits a sum in FP32 error-free transformations:
//   t_k = q_k - x_k = th + tl exactly (TwoSum);  th^2 = p + pe exactly (FMA);
//   t_k^2 = p + (pe + 2 th tl) + tl^2, with tl^2 <= 2^-48 th^2 dropped;
//   the p_k are added with TwoSum, whose errors are collected in FP32 (c), and the small
//   parts m_k = fl(pe + fl(2 th tl)) in FP32 (m).
// For non-negative terms every TwoSum error is at most 2^-24 of the whole sum, at most d-1 of
// them are non-zero, and every FP32 sum here has at most d+32 roundings on any path, so with
// S = (s + c) + m in FP64:
//   |S - D| <= [(d+32)(d-1) + 3(d+32) + 6 + 1/16] 2^-48 D (1 + 2^-20) + 4d 2^-150
//           <= (d+34)^2 2^-48 D + (d+1) 2^-146
// (the 2^-150 terms are the roundings of products and sums that fall below the normal range).
// The _rn intrinsics are never contracted into FMAs, so each step rounds exactly once.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}

struct FFSum {
    float s;   // TwoSum chain of the p_k
    float c;   // its collected errors
    float m;   // the small parts
};

__device__ __forceinline__ void ff_add_term(FFSum &a, float q, float x)
{
    float th, tl;
    two_sum(q, -x, th, tl);
    const float p = __fmul_rn(th, th);
    const float pe = __fmaf_rn(th, th, -p);
    a.m = __fadd_rn(a.m, __fadd_rn(pe, __fmul_rn(__fadd_rn(th, th), tl)));
    float s, e;
    two_sum(a.s, p, s, e);
    a.s = s;
    a.c = __fadd_rn(a.c, e);
}

__device__ __forceinline__ void ff_merge(FFSum &a, float bs, float bc, float bm)
{
    float s, e;
    two_sum(a.s, bs, s, e);
    a.s = s;
    a.c = __fadd_rn(__fadd_rn(a.c, bc), e);
    a.m = __fadd_rn(a.m, bm);
}

// Float-float value S of sum_k (q_k - x_k)^2 by the whole warp (lane l takes k = l, l+32, ...;
// a butterfly of commutative merges, so every lane returns the same S).
__device__ __forceinline__ double warp_ff_sq(const float *__restrict__ q, const float *__restrict__ x, int d)
{
    const unsigned lane = threadIdx.x & 31;
    FFSum a{0.f, 0.f, 0.f};
    for (int k = (int)lane; k < d; k += 32) ff_add_term(a, __ldg(q + k), __ldg(x + k));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        ff_merge(a, __shfl_xor_sync(0xffffffffu, a.s, o), __shfl_xor_sync(0xffffffffu, a.c, o),
                 __shfl_xor_sync(0xffffffffu, a.m, o));
    return __dadd_rn(__dadd_rn((double)a.s, (double)a.c), (double)a.m);
}

// Thresholds of the float-float stage for eps^2 = e2: accept if S <= t_acc (then
// D <= e2 (1 - g64), so the canonical value C <= D (1 + g64) < e2), reject if S > t_rej (then
// D > e2 (1 + 2 g64) and C >= D (1 - g64) > e2), with g64 = (d+4) 2^-53 the canonical sum's
// relative error. Every factor is exact in FP64 and every operation rounds outward.
__device__ __forceinline__ void ff_thresholds(double e2, int d, double *t_acc, double *t_rej)
{
    const double g64 = (double)(d + 4) * 0x1p-53;
    const double dd = (double)(d + 34);
    const double del = dd * dd * 0x1p-48;
    const double abs_ff = (double)(d + 1) * 0x1p-146;
    *t_acc = __dsub_rd(__dmul_rd(__dmul_rd(e2, 1.0 - g64), 1.0 - del), abs_ff);
    *t_rej = __dadd_ru(__dmul_ru(__dmul_ru(e2, 1.0 + 2.0 * g64), 1.0 + del), abs_ff);
}

// FP32 squared distance of (q, x) computed by the whole warp: each lane sums a slice
// (16-byte loads when d % 4 == 0: store rows are then 16-byte aligned), then a shuffle
// tree. Every lane returns the sum. The (d+8) 2^-24 bound of fp32_thresholds holds for
// any summation order.
__device__ __forceinline__ float warp_sq32(const float *__restrict__ q, const float *__restrict__ x, int d)
{
    const unsigned lane = threadIdx.x & 31;
    float s = 0.f;
    if ((d & 3) == 0) {
        const float4 *q4 = reinterpret_cast<const float4 *>(q);
        const float4 *x4 = reinterpret_cast<const float4 *>(x);
        for (int k = lane; k < (d >> 2); k += 32) {
            const float4 a = __ldg(q4 + k), b = __ldg(x4 + k);
            float t = a.x - b.x;
            s = fmaf(t, t, s);
            t = a.y - b.y;
            s = fmaf(t, t, s);
            t = a.z - b.z;
            s = fmaf(t, t, s);
            t = a.w - b.w;
            s = fmaf(t, t, s);
        }
    } else {
        for (int k = lane; k < d; k += 32) {
            const float t = __ldg(q + k) - __ldg(x + k);
            s = fmaf(t, t, s);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// The canonical FP64 sum of (q, x) by the whole warp: lane l forms the term of dimension
// k0 + l, then lane 0 adds the terms in ascending k with __dadd_rn, so the sum is exactly the
// sequential definition's. Every lane returns it.
__device__ __forceinline__ double warp_canonical64(const float *__restrict__ q, const float *__restrict__ x, int d)
{
    const unsigned lane = threadIdx.x & 31;
    double sum = 0.0;
    for (int k0 = 0; k0 < d; k0 += 32) {
        double pk = 0.0;
        const int k = k0 + (int)lane;
        if (k < d) {
            const double t = __dsub_rn((double)__ldg(q + k), (double)__ldg(x + k));
            pk = __dmul_rn(t, t);
        }
        const int lim = min(32, d - k0);
        for (int l = 0; l < lim; ++l) {
            const double v = __shfl_sync(0xffffffffu, pk, l);
            if (lane == 0) sum = __dadd_rn(sum, v);   // one lane runs the chain: the FP64 rate is low
        }
    }
    return __shfl_sync(0xffffffffu, sum, 0);
}

// Exact decision for the pair (q, x), taken by the whole warp (same answer in
// every lane): FP32 first, then the float-float sum, the canonical FP64 sum only when
// neither can decide.
__device__ __forceinline__ bool warp_exact_decide(const float *__restrict__ q, const float *__restrict__ x, int d,
                                                  double e2, float t_acc, float t_rej,
                                                  unsigned long long *__restrict__ n_fp64)
{
    const float s = warp_sq32(q, x, d);
    if (s <= t_acc) return true;
    if (s > t_rej) return false;
    double fa, fr;
    ff_thresholds(e2, d, &fa, &fr);
    const double sf = warp_ff_sq(q, x, d);
    if (sf <= fa) return true;
    if (sf > fr) return false;
    const double sum = warp_canonical64(q, x, d);
    if ((threadIdx.x & 31) == 0) atomicAdd(n_fp64, 1ULL);
    return sum <= e2;
}

// Exact decisions for the band entries among a warp's 32 candidate entries. Each lane in
// bm holds a band pair (q, x) with its own squared threshold e2 and FP32 thresholds. Four
// pairs are settled at a time, one per 8-lane group: the group sums the pair's FP32
// squared distance over 16-byte slices (a shuffle tree within the group; the (d+8) 2^-24
// bound holds for any order) and compares it with the pair's thresholds. The pairs that
// FP32 cannot decide are then settled one by one by the whole warp with the float-float
// sum, and the few that it cannot place either with the canonical FP64 sum. Returns this
// lane's decision (false for lanes not in bm); *used_fp64 is set in the lanes whose pair
// needed the canonical FP64 sum.
__device__ __forceinline__ bool warp_band_decide(unsigned bm, const float *q, const float *x, int d, double e2,
                                                 float t_acc, float t_rej, bool *used_fp64)
{
    const unsigned lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const int grp = (int)(lane >> 3), gl = (int)(lane & 7);
    bool mine = false, und = false;
    unsigned rem = bm;
    while (rem) {
        const unsigned pos = __fns(rem, 0, grp + 1);   // this group's entry: the (grp+1)-th pending lane
        const bool have = pos < 32u;
        const int k = have ? (int)pos : 0;
        const float *qk = reinterpret_cast<const float *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(q), k));
        const float *xk = reinterpret_cast<const float *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(x), k));
        float s = 0.f;
        if (have) {
            if ((d & 3) == 0) {
                // four 16-byte slices of each row in flight per lane (zero past the row: adds 0)
                const float4 *q4 = reinterpret_cast<const float4 *>(qk);
                const float4 *x4 = reinterpret_cast<const float4 *>(xk);
                const int n4 = d >> 2;
                for (int i0 = gl; i0 < n4; i0 += 32) {
                    float4 a[4], b[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int i = i0 + 8 * u;
                        a[u] = i < n4 ? __ldg(q4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
                        b[u] = i < n4 ? __ldg(x4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        float t = a[u].x - b[u].x;
                        s = fmaf(t, t, s);
                        t = a[u].y - b[u].y;
                        s = fmaf(t, t, s);
                        t = a[u].z - b[u].z;
                        s = fmaf(t, t, s);
                        t = a[u].w - b[u].w;
                        s = fmaf(t, t, s);
                    }
                }
            } else {
                for (int i = gl; i < d; i += 8) {
                    const float t = __ldg(qk + i) - __ldg(xk + i);
                    s = fmaf(t, t, s);
                }
            }
        }
        s += __shfl_xor_sync(0xffffffffu, s, 4);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        const float ta = __shfl_sync(0xffffffffu, t_acc, k);
        const float tr = __shfl_sync(0xffffffffu, t_rej, k);
        const unsigned accm = __ballot_sync(0xffffffffu, have && gl == 0 && s <= ta);
        const unsigned undm = __ballot_sync(0xffffffffu, have && gl == 0 && !(s <= ta) && !(s > tr));
        if ((rem >> lane) & 1u) {   // an entry of this round: rank r among the pending lanes
            const int r = __popc(rem & below);
            if (r < 4) {
                mine = ((accm >> (8 * r)) & 1u) != 0u;
                und = ((undm >> (8 * r)) & 1u) != 0u;
            }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) rem &= rem - 1u;   // the four settled entries leave the set
    }
    bool f64 = false;
    unsigned um = __ballot_sync(0xffffffffu, und);
    while (um) {   // one by one, the whole warp: the float-float sum, then the canonical one
        const int k = __ffs(um) - 1;
        um &= um - 1u;
        const float *qk = reinterpret_cast<const float *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(q), k));
        const float *xk = reinterpret_cast<const float *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(x), k));
        const double e2k = __shfl_sync(0xffffffffu, e2, k);
        double fa, fr;
        ff_thresholds(e2k, d, &fa, &fr);
        const double sf = warp_ff_sq(qk, xk, d);
        bool dec = sf <= fa;
        if (!dec && !(sf > fr)) {
            dec = warp_canonical64(qk, xk, d) <= e2k;
            if ((int)lane == k) f64 = true;
        }
        if ((int)lane == k) mine = dec;
    }
    *used_fp64 = f64;
    return mine;
}

// The canonical FP64 dot product of (q, x) by the whole warp: lane l forms the (exact) product
// of dimension k0 + l, lane 0 adds the products in ascending k with __dadd_rn -- the
// sequential definition. Every lane returns it.
__device__ __forceinline__ double warp_canonical_dot(const float *__restrict__ q, const float *__restrict__ x, int d)
{
    const unsigned lane = threadIdx.x & 31;
    double sum = 0.0;
    for (int k0 = 0; k0 < d; k0 += 32) {
        double pk = 0.0;
        const int k = k0 + (int)lane;
        if (k < d) pk = __dmul_rn((double)__ldg(q + k), (double)__ldg(x + k));   // exact: 24 x 24 bits
        const int lim = min(32, d - k0);
        for (int l = 0; l < lim; ++l) {
            const double v = __shfl_sync(0xffffffffu, pk, l);
            if (lane == 0) sum = __dadd_rn(sum, v);
        }
    }
    return __shfl_sync(0xffffffffu, sum, 0);
}

// Exact decisions of the inner-product join's band entries (q.x >= t by the canonical FP64
// dot), one 8-lane group per pair as in warp_band_decide: the FP32 dot S32 and A32 =
// sum |q_k x_k| over 16-byte slices; with B = cf A32 + ca (which covers the FP32 error, the
// canonical dot's own error and A32's rounding), accept if RD(S32 - B) >= t_ru (then the
// canonical dot is >= t), reject if RU(S32 + B) < t_rd, else the canonical FP64 dot decides.
// t_ru / t_rd: t rounded up / down to FP32. *used_fp64 marks the lanes that needed it.
__device__ __forceinline__ bool warp_band_decide_ip(unsigned bm, const float *q, const float *x, int d, double t,
                                                    float t_ru, float t_rd, float cf, float ca, bool *used_fp64)
{
    const unsigned lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const int grp = (int)(lane >> 3), gl = (int)(lane & 7);
    bool mine = false, und = false;
    unsigned rem = bm;
    while (rem) {
        const unsigned pos = __fns(rem, 0, grp + 1);
        const bool have = pos < 32u;
        const int k = have ? (int)pos : 0;
        const float *qk = reinterpret_cast<const float *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(q), k));
        const float *xk = reinterpret_cast<const float *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(x), k));
        float sd = 0.f, sa = 0.f;
        if (have) {
            if ((d & 3) == 0) {
                const float4 *q4 = reinterpret_cast<const float4 *>(qk);
                const float4 *x4 = reinterpret_cast<const float4 *>(xk);
                const int n4 = d >> 2;
                for (int i = gl; i < n4; i += 8) {
                    const float4 a = __ldg(q4 + i), b = __ldg(x4 + i);
                    sd = fmaf(a.x, b.x, sd);
                    sa = fmaf(fabsf(a.x), fabsf(b.x), sa);
                    sd = fmaf(a.y, b.y, sd);
                    sa = fmaf(fabsf(a.y), fabsf(b.y), sa);
                    sd = fmaf(a.z, b.z, sd);
                    sa = fmaf(fabsf(a.z), fabsf(b.z), sa);
                    sd = fmaf(a.w, b.w, sd);
                    sa = fmaf(fabsf(a.w), fabsf(b.w), sa);
                }
            } else {
                for (int i = gl; i < d; i += 8) {
                    const float a = __ldg(qk + i), b = __ldg(xk + i);
                    sd = fmaf(a, b, sd);
                    sa = fmaf(fabsf(a), fabsf(b), sa);
                }
            }
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            sd += __shfl_xor_sync(0xffffffffu, sd, o);
            sa += __shfl_xor_sync(0xffffffffu, sa, o);
        }
        const float bnd = __fmaf_ru(cf, sa, ca);
        const bool accept = __fsub_rd(sd, bnd) >= t_ru;
        const bool reject = __fadd_ru(sd, bnd) < t_rd;
        const unsigned accm = __ballot_sync(0xffffffffu, have && gl == 0 && accept);
        const unsigned undm = __ballot_sync(0xffffffffu, have && gl == 0 && !accept && !reject);
        if ((rem >> lane) & 1u) {
            const int r = __popc(rem & below);
            if (r < 4) {
                mine = ((accm >> (8 * r)) & 1u) != 0u;
                und = ((undm >> (8 * r)) & 1u) != 0u;
            }
        }
#pragma unroll
        for (int tt = 0; tt < 4; ++tt) rem &= rem - 1u;
    }
    *used_fp64 = und;
    unsigned um = __ballot_sync(0xffffffffu, und);
    while (um) {
        const int k = __ffs(um) - 1;
        um &= um - 1u;
        const float *qk = reinterpret_cast<const float *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(q), k));
        const float *xk = reinterpret_cast<const float *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(x), k));
        const bool dec = warp_canonical_dot(qk, xk, d) >= t;
        if ((int)lane == k) mine = dec;
    }
    return mine;
}

// Warp-aggregated atomicAdd of `v` to counter[key]: lanes with equal keys are
// grouped (__match_any_sync), the group's lowest lane adds the group's total and
// every lane gets its own offset. Every lane of the warp must call it; lanes
// with active == false add nothing.
__device__ __forceinline__ unsigned long long grouped_add(unsigned long long *counter, int key, bool active,
                                                          unsigned v)
{
    const unsigned lane = threadIdx.x & 31;
    const unsigned act = __ballot_sync(0xffffffffu, active);
    unsigned long long off = 0;
    if (active) {
        const unsigned peers = __match_any_sync(act, key);
        const int leader = __ffs(peers) - 1;
        const unsigned below = peers & ((1u << lane) - 1u);
        // prefix of v over the lower peers (v is 1 for every caller here, so popc)
        unsigned long long base = 0;
        if ((int)lane == leader) base = atomicAdd(counter + key, (unsigned long long)(__popc(peers) * v));
        base = __shfl_sync(peers, base, leader);
        off = base + (unsigned long long)__popc(below) * v;
    }
    return off;
}

}  // namespace dl
