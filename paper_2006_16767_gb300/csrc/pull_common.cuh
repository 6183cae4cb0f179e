// Definitions shared by the row-major (pull) kernels.
#pragma once
#include <type_traits>

#include "internal.h"
#include "prims.cuh"

namespace asv {

template <class T>
__device__ __forceinline__ T __int_as_float_t(int v) {
    if constexpr (sizeof(T) == 4 && std::is_same<T, float>::value) return __int_as_float(v);
    else return (T)v;
}

struct PullArg {
    const CallDesc* desc;  // read x/y from the call descriptor when non-null
    PullIO io;             // otherwise the pointers given directly
};

__device__ __forceinline__ PullIO resolve(const PullArg& a, void* ywork, bool sparse_out) {
    if (a.desc) {
        PullIO p;
        p.x = a.desc->x_dense;
        p.xbits = a.desc->xbits;
        p.y = sparse_out ? ywork : a.desc->y;
        p.ymask = a.desc->ymask;
        return p;
    }
    return a.io;
}

// The first-term-then-four-per-step Boolean walk of entries [b, e) of one
// row by one lane: the first term alone (with a dense frontier most rows stop
// there), then four terms per step with their index loads and bit gathers in
// flight together; OR is settled by the first true term.
__device__ __forceinline__ uint32_t bool_walk(const int32_t* __restrict__ col, const bool8* __restrict__ x,
                                              const uint32_t* __restrict__ xbits, int32_t b, int32_t e) {
    if (b < e && bool_gather(x, xbits, __ldg(col + b))) return 1u;
    for (int32_t k = b + 1; k < e; k += 4) {
        int32_t c[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) c[u] = k + u < e ? __ldg(col + k + u) : -1;
        uint32_t t = 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u) t |= c[u] >= 0 ? bool_gather(x, xbits, c[u]) : 0u;
        if (t) return 1u;
    }
    return 0u;
}

// One row per thread in the (OR, AND) semiring: the warp's 32 rows r0 ..
// r0 + 31 (rows of more than kLongRow entries are left to the long-row
// pass, rows the output mask excludes give 0). Each lane walks the first
// kAlone entries of its row alone (bool_walk); a row still undecided after
// them would hold the whole warp for a serial chain of loads, so the warp
// finishes those rows together, 64 terms (two coalesced index loads and
// their bit gathers) per step. Writes y (dense output) or, for a sparse
// output, the row's flag when it has a true term.
template <bool SOUT>
__device__ __forceinline__ void pull_rows_bool(int64_t m, const int32_t* __restrict__ rowptr,
                                               const int32_t* __restrict__ col, const PullIO& p, bool8* y,
                                               uint8_t* yflag, int64_t r0, int lane) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int32_t kAlone = 32;
    const bool8* __restrict__ x = (const bool8*)p.x;
    const int64_t i = r0 + lane;
    const int32_t rb = __ldg(rowptr + min(i, m));
    const int32_t span_end = __ldg(rowptr + min(r0 + 32, m));
    const int32_t re_n = __shfl_down_sync(FULL, rb, 1);
    const int32_t re = (lane == 31) ? span_end : re_n;
    const bool mine = i < m && re - rb <= kLongRow;
    const bool on = mine && !row_masked(p.ymask, i);
    uint32_t acc = on ? bool_walk(col, x, p.xbits, rb, min(re, rb + kAlone)) : 0u;
    const bool coop = on && !acc && re - rb > kAlone;
    for (unsigned pend = __ballot_sync(FULL, coop); pend; pend &= pend - 1) {
        const int src = __ffs(pend) - 1;
        const int32_t b = __shfl_sync(FULL, rb, src) + kAlone, e = __shfl_sync(FULL, re, src);
        bool found = false;
        for (int32_t k0 = b; k0 < e && !found; k0 += 64) {
            const int32_t k1 = k0 + lane, k2 = k0 + 32 + lane;
            const int32_t c1 = k1 < e ? __ldg(col + k1) : -1, c2 = k2 < e ? __ldg(col + k2) : -1;
            const uint32_t t = (c1 >= 0 ? bool_gather(x, p.xbits, c1) : 0u) |
                               (c2 >= 0 ? bool_gather(x, p.xbits, c2) : 0u);
            found = __any_sync(FULL, t != 0u);
        }
        if (lane == src && found) acc = 1u;
    }
    if (mine) {
        // a Boolean sparse output is its flags (the emitted values are one)
        if (!SOUT) y[i] = (bool8)acc;
        if (SOUT && acc) yflag[i] = 1;
    }
}

}  // namespace asv
