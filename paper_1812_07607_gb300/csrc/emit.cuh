// emit.cuh -- warp-aggregated compaction of join output (K5).
//
// A warp that has matches in one step ballots them, its lane 0 reserves room
// for all of them with ONE atomicAdd on the global counter, and every matching
// lane writes at base + (number of matching lanes below it). Positions at or
// past the capacity are counted but not written, so the host can detect an
// overflow and size a re-run exactly.
#pragma once

#include <cstdint>

namespace dl {

struct JoinOut {
    const int64_t *r_ids;          // ids of the R store
    const int64_t *s_ids;          // ids of the S store (== r_ids for a self-join)
    int64_t *out_r;                // [out_cap] pair ids, R side
    int64_t *out_s;                // [out_cap] pair ids, S side
    unsigned long long *out_cnt;   // pairs produced (may exceed out_cap)
    unsigned long long out_cap;
    uint2 *band;                   // [band_cap] (r row, s row) pairs left for the recheck
    unsigned long long *band_cnt;
    unsigned long long band_cap;
    int mirror;                    // 1: self-join full mode, also write (s, r)
    const int32_t *orig;           // self-join upper mode: caller's row index per store row, so that
                                   // each unordered pair is written (lower caller row, higher); else NULL
};

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Every lane of the warp must call this (it ballots). `acc` / `band` say whether
// the calling lane's pair (r, c) is a proven match / an undecided band pair.
__device__ __forceinline__ void warp_emit(const JoinOut &o, bool acc, bool band, int r, int c)
{
    const unsigned am = __ballot_sync(0xffffffffu, acc);
    const unsigned bm = __ballot_sync(0xffffffffu, band);
    const unsigned lt = lanemask_lt();
    const unsigned lane = threadIdx.x & 31;
    if (am) {
        const unsigned mult = o.mirror ? 2u : 1u;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(o.out_cnt, (unsigned long long)(__popc(am) * mult));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (acc) {
            const unsigned long long pos = base + (unsigned long long)(__popc(am & lt) * mult);
            int64_t ri = o.r_ids[r], si = o.s_ids[c];
            if (o.orig && o.orig[r] > o.orig[c]) {
                const int64_t tmp = ri;
                ri = si;
                si = tmp;
            }
            if (pos < o.out_cap) {
                o.out_r[pos] = ri;
                o.out_s[pos] = si;
            }
            if (mult == 2 && pos + 1 < o.out_cap) {
                o.out_r[pos + 1] = si;
                o.out_s[pos + 1] = ri;
            }
        }
    }
    if (bm) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(o.band_cnt, (unsigned long long)__popc(bm));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (band) {
            const unsigned long long pos = base + (unsigned long long)__popc(bm & lt);
            if (pos < o.band_cap) o.band[pos] = make_uint2((unsigned)r, (unsigned)c);
        }
    }
}

}  // namespace dl
