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
        p.y = sparse_out ? (a.desc->y_ident ? a.desc->yval : ywork) : a.desc->y;
        p.ymask = a.desc->ymask;
        return p;
    }
    return a.io;
}

// Groups of 32 rows per warp in the (OR, AND) thread pull: each lane walks
// one row of every group, the groups' loads interleaved, so a warp keeps
// twice the loads in flight that one row per lane would.
constexpr int kBoolRows = 2;

// One row per thread in the (OR, AND) semiring: the warp's 32 * kBoolRows
// rows r0 .. (lane l takes rows r0 + 32 g + l), rows of more than kLongRow
// entries left to the long-row pass, rows the output mask excludes giving 0.
// Each lane walks the first kAlone entries of its rows alone -- the first
// terms of all its rows together (with a dense frontier most rows stop
// there), then four terms of each undecided row per step, every index load
// and bit gather of a step in flight together; OR is settled by the first
// true term. A row still undecided after them would hold the whole warp for
// a serial chain of loads, so the warp finishes those rows together, 64
// terms (two coalesced index loads and their bit gathers) per step. Writes
// y (dense output) or, for a sparse output, the row's flag when it has a
// true term.
template <bool SOUT>
__device__ __forceinline__ void pull_rows_bool(int64_t m, const int32_t* __restrict__ rowptr,
                                               const int32_t* __restrict__ col, const PullIO& p, bool8* y,
                                               uint8_t* yflag, int64_t r0, int lane) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int32_t kAlone = 32;
    constexpr int R = kBoolRows;
    const bool8* __restrict__ x = (const bool8*)p.x;
    int32_t rb[R], re[R];
    bool mine[R], on[R];
    uint32_t acc[R];
#pragma unroll
    for (int g = 0; g < R; ++g) rb[g] = __ldg(rowptr + min(r0 + 32 * g + lane, m));
    const int32_t tail = __ldg(rowptr + min(r0 + 32 * R, m));
#pragma unroll
    for (int g = 0; g < R; ++g) {
        const int32_t nx = __shfl_down_sync(FULL, rb[g], 1);
        const int32_t first_next = (g + 1 < R) ? __shfl_sync(FULL, rb[g + 1 < R ? g + 1 : g], 0) : tail;
        re[g] = (lane == 31) ? first_next : nx;
        const int64_t i = r0 + 32 * g + lane;
        mine[g] = i < m && re[g] - rb[g] <= kLongRow;
        on[g] = mine[g] && !row_masked(p.ymask, i);
    }
    int32_t c0[R];
#pragma unroll
    for (int g = 0; g < R; ++g) c0[g] = (on[g] && rb[g] < re[g]) ? __ldg(col + rb[g]) : -1;
#pragma unroll
    for (int g = 0; g < R; ++g) acc[g] = c0[g] >= 0 ? bool_gather(x, p.xbits, c0[g]) : 0u;
    int32_t k[R], lim[R];
#pragma unroll
    for (int g = 0; g < R; ++g) {
        k[g] = rb[g] + 1;
        lim[g] = min(re[g], rb[g] + kAlone);
    }
    for (;;) {
        int32_t cc[R][4];
        bool any = false;
#pragma unroll
        for (int g = 0; g < R; ++g) {
            const bool act = on[g] && !acc[g] && k[g] < lim[g];
            any |= act;
#pragma unroll
            for (int u = 0; u < 4; ++u) cc[g][u] = (act && k[g] + u < lim[g]) ? __ldg(col + k[g] + u) : -1;
        }
        if (!any) break;
#pragma unroll
        for (int g = 0; g < R; ++g) {
            uint32_t t = 0u;
#pragma unroll
            for (int u = 0; u < 4; ++u) t |= cc[g][u] >= 0 ? bool_gather(x, p.xbits, cc[g][u]) : 0u;
            acc[g] |= t;
            k[g] += 4;
        }
    }
#pragma unroll
    for (int g = 0; g < R; ++g) {
        const bool coop = on[g] && !acc[g] && re[g] - rb[g] > kAlone;
        for (unsigned pend = __ballot_sync(FULL, coop); pend; pend &= pend - 1) {
            const int src = __ffs(pend) - 1;
            const int32_t b = __shfl_sync(FULL, rb[g], src) + kAlone, e = __shfl_sync(FULL, re[g], src);
            bool found = false;
            for (int32_t k0 = b; k0 < e && !found; k0 += 64) {
                const int32_t k1 = k0 + lane, k2 = k0 + 32 + lane;
                const int32_t c1 = k1 < e ? __ldg(col + k1) : -1, c2 = k2 < e ? __ldg(col + k2) : -1;
                const uint32_t t = (c1 >= 0 ? bool_gather(x, p.xbits, c1) : 0u) |
                                   (c2 >= 0 ? bool_gather(x, p.xbits, c2) : 0u);
                found = __any_sync(FULL, t != 0u);
            }
            if (lane == src && found) acc[g] = 1u;
        }
        const int64_t i = r0 + 32 * g + lane;
        if (mine[g]) {
            // a Boolean sparse output is its flags (the emitted values are one)
            if (!SOUT) y[i] = (bool8)acc[g];
            if (SOUT && acc[g]) yflag[i] = 1;
        }
    }
}

}  // namespace asv
