// checked.cuh -- the bounds-checked build (compiled with -DDL_CHECKED).
//
// DL_CHECK(cond, site, index) guards a computed shared- or global-memory access. In the
// checked build it evaluates `cond`; when that fails it records the first failure of the
// translation unit -- the site code and the offending index -- in a device word and yields
// false, so the caller skips the access instead of faulting (nothing traps). In the normal
// build it is the constant true and costs nothing. Each translation unit that uses it holds
// its own word (no relocatable device code is needed); DL_CHECK_READER(unit) defines the host
// function that reads and clears it, and dl_debug_check_word() gathers every unit's word.
#pragma once

#include <cstdint>

#ifdef DL_CHECKED

namespace dl {
// (site << 40) | (index & (2^40 - 1)) of this translation unit's first failed check; 0 = none.
static __device__ unsigned long long g_check_word;

__device__ __forceinline__ bool check_ok(bool ok, unsigned site, long long index)
{
    if (!ok)
        atomicCAS(&g_check_word, 0ull,
                  ((unsigned long long)site << 40) | ((unsigned long long)index & 0xFFFFFFFFFFull));
    return ok;
}
}  // namespace dl

#define DL_CHECK(cond, site, index) ::dl::check_ok((cond), (site), (long long)(index))

// Host reader of this unit's word (reads, then clears it); returns a cudaError_t.
#define DL_CHECK_READER(unit)                                                                      \
    namespace dl {                                                                                 \
    int check_read_##unit(unsigned long long *out)                                                 \
    {                                                                                              \
        unsigned long long zero = 0;                                                               \
        cudaError_t e = cudaMemcpyFromSymbol(out, g_check_word, sizeof zero);                      \
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_check_word, &zero, sizeof zero);            \
        return (int)e;                                                                             \
    }                                                                                              \
    }

#else

#define DL_CHECK(cond, site, index) true
#define DL_CHECK_READER(unit)                                                                      \
    namespace dl {                                                                                 \
    int check_read_##unit(unsigned long long *out)                                                 \
    {                                                                                              \
        *out = 0;                                                                                  \
        return 0;                                                                                  \
    }                                                                                              \
    }

#endif
