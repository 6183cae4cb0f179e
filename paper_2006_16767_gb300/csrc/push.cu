// Column-major ("push") SpMSpV candidates, solution (2,8) of Sec. IV-A: for
// every listed nonzero x_j, the entries of column j (CSC) are scaled by x_j
// and written back into y. Workload distribution (Sec. IV-B): one listed
// column per thread (the paper's "direct"), one warp per column, or an even
// split of the effective nonzeros (merge-based, after Yang et al.). Write-back
// (Sec. IV-B): atomic accumulation (one kernel), sort-based ((row, value)
// pairs to memory, radix sort by row, reduce-by-key), or privatised
// accumulation of row tiles in shared memory after bucketing the pairs.
//
// Accumulation of the floating-point types is in FP64 (products are formed in
// the value type), so the order in which atomics land does not move an FP32
// result by more than one rounding -- except on FP32 matrices whose rows all
// have at most kNarrowRow entries, whose atomics for a dense output add in
// FP32 (WB_ATOM_N):
// y_i then sums at most k <= 32 products, and k FP32 products added in any
// order stay within k * 2^-24 * sum |a_ij x_j| <= 1.91e-6 * sum |a_ij x_j| of
// the exact sum (the FP32 tolerance is 2e-6 of it); those atomics add
// straight into the zeroed output, with no accumulator to write out.
#include "internal.h"
#include "prims.cuh"
#include "sort.cuh"

namespace asv {

enum { WB_ATOM = 0, WB_SORT = 1, WB_PRIV = 2, WB_ATOM_N = 3 };
__host__ __device__ constexpr bool wb_atomic(int wb) { return wb == WB_ATOM || wb == WB_ATOM_N; }
constexpr int kPrivBits = 12;  // rows per privatised tile = 4096
constexpr int kPushIPT = 8;    // effective nonzeros per lane per balanced chunk

template <class T>
using PV = typename std::conditional<sizeof(T) == 8, uint64_t, uint32_t>::type;

// One effective nonzero (row r, product p) at effective index pos.
template <class T, int WB>
__device__ __forceinline__ void emit(const Ws& ws, const uint32_t* ymask, int32_t r, typename Sr<T>::Part p,
                                     int64_t pos) {
    using S = Sr<T>;
    if (wb_atomic(WB)) {
        if (row_masked(ymask, r)) return;  // excluded by the output mask (pairs are masked when reduced)
        if constexpr (!S::kPattern) {
            if constexpr (WB == WB_ATOM_N) {
                // straight into the dense output, zeroed before the push: no
                // flag (a dense output needs no structural set)
                atomicAdd((T*)ws.acc + r, S::part_T(p));
            } else {
                atomicAdd((typename S::Atom*)ws.acc + r, S::to_atom(S::part_T(p)));
                ws.yflag[r] = 1;
            }
        } else {
            // a Boolean search reaches most rows many times: a (possibly
            // L1-stale) read that already sees the flag saves the store; a
            // stale 0 only costs one
            if (ws.yflag[r] == 0) ws.yflag[r] = 1;
        }
    } else {
        ws.pkeys[0][pos] = (uint32_t)r;
        if constexpr (!S::kPattern) {
            const T v = S::part_T(p);
            ((T*)ws.pvals[0])[pos] = v;
        }
    }
}

// N write-backs of one thread (rows r[u] < 0 are skipped; item u's
// effective index is pos0 + u * pstride). For a Boolean atomic write-back
// all the flag reads are issued before any store.
template <class T, int WB, int N>
__device__ __forceinline__ void emit_batch(const Ws& ws, const uint32_t* ymask, const int32_t (&r)[N],
                                           const typename Sr<T>::Part (&p)[N], int64_t pos0, int64_t pstride) {
    if constexpr (wb_atomic(WB) && Sr<T>::kPattern) {
        uint8_t f[N];
#pragma unroll
        for (int u = 0; u < N; ++u) f[u] = r[u] >= 0 ? ws.yflag[r[u]] : (uint8_t)1;
#pragma unroll
        for (int u = 0; u < N; ++u)
            if (!f[u] && !row_masked(ymask, r[u])) ws.yflag[r[u]] = 1;
    } else {
#pragma unroll
        for (int u = 0; u < N; ++u)
            if (r[u] >= 0) emit<T, WB>(ws, ymask, r[u], p[u], pos0 + u * pstride);
    }
}

// N write-backs of one thread at the effective indexes pos[u] (rows r[u] < 0
// are skipped; effective indexes are those of the 32-bit list scan), the
// Boolean flag reads again issued before any store.
template <class T, int WB, int N>
__device__ __forceinline__ void emit_slots(const Ws& ws, const uint32_t* ymask, const int32_t (&r)[N],
                                           const typename Sr<T>::Part (&p)[N], const int32_t (&pos)[N]) {
    if constexpr (wb_atomic(WB) && Sr<T>::kPattern) {
        emit_batch<T, WB, N>(ws, ymask, r, p, 0, 0);
    } else {
#pragma unroll
        for (int u = 0; u < N; ++u)
            if (r[u] >= 0) emit<T, WB>(ws, ymask, r[u], p[u], pos[u]);
    }
}

// The workspaces a push kernel writes through: with FP32 accumulation for a
// dense output (WB_ATOM_N) the accumulators are the output itself.
template <int WB>
__device__ __forceinline__ Ws push_ws(Ws w, const CallDesc* d) {
    if constexpr (WB == WB_ATOM_N) w.acc = d->y;
    return w;
}

// Zeroes the dense output ahead of a push that accumulates into it (16-byte
// stores from the first aligned element).
template <class T>
__global__ void __launch_bounds__(256) k_zero_out(int64_t m, const CallDesc* __restrict__ desc, Gate gate) {
    if (gate.off()) return;
    T* __restrict__ y = (T*)desc->y;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
    constexpr int64_t V = 16 / sizeof(T);
    const int64_t head = min(m, (int64_t)(((16 - ((uintptr_t)y & 15)) & 15) / sizeof(T)));
    if (tid < head) y[tid] = T(0);
    const int64_t nv = (m - head) / V;
    uint4* __restrict__ yv = reinterpret_cast<uint4*>(y + head);
    for (int64_t i = tid; i < nv; i += nt) yv[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int64_t i = head + nv * V + tid; i < m; i += nt) y[i] = T(0);
}

template <class T>
__device__ __forceinline__ T list_val(const CallDesc* d, int64_t t) {
    if (Sr<T>::kPattern || d->xval == nullptr) return Sr<T>::one();
    return ((const T*)d->xval)[t];
}

// ---------------------------------------------------------------- traversals
// One listed column per thread for columns of at most kLongCol entries; a
// longer column (a hub of a power-law graph can hold 10^5 entries) is walked
// by its whole warp right after, so no thread serialises a hub alone.
constexpr int kLongCol = 64;

// A listed column of more than kLongSeg entries (a hub) would keep one warp
// busy long after the rest of the grid is done, so the warp that meets it
// queues it instead, and every warp, once its own columns are done, takes
// segments of kLongSeg entries from the queued columns through per-column
// atomic cursors. The warp that queued a column reaches the queue after
// queuing it, so every segment is taken whatever the other warps do. The
// feature pass counted the list's hubs (desc->nhub), so in the thread push,
// where a short list of hubs leaves nearly the whole grid without columns of
// its own, a warp first waits, for a bounded time, until that many are
// queued; without the wait it would find the queue still empty and leave the
// hubs to the one or two warps that own them (37 hub columns of 6.8M entries:
// 36 ms instead of 0.6 ms). The warp push does not wait: there every listed
// column has its own warp, and on the same list its 37 owner warps sweeping
// the queued columns together (0.25 ms) beat the whole grid joining them
// (0.58 ms): the owners take the queued columns one after the other, so the
// segments in flight at a time are consecutive ones of one column, on
// disjoint rows. The wait only decides who helps, never what is done.
constexpr int kHubWaitIters = 256;  // x ~128 ns of sleep: a few tens of microseconds at most
template <class T, int WB>
__device__ __forceinline__ void push_segment(const int32_t* __restrict__ colptr, const int32_t* __restrict__ rowidx,
                                             const T* __restrict__ valc, const CallDesc* __restrict__ desc,
                                             const Ws& ws, const uint32_t* ym, int64_t t, int32_t s, int lane,
                                             bool bm) {
    using S = Sr<T>;
    // bm: t is the column itself (a dense x read from its bitmap, no list)
    const int32_t j = bm ? (int32_t)t : desc->xidx[t];
    T xj = S::one();
    if constexpr (!S::kPattern) xj = bm ? ((const T*)desc->x_dense)[j] : list_val<T>(desc, t);
    const int32_t b = __ldg(colptr + j), e = __ldg(colptr + j + 1);
    const int64_t pos0 = !wb_atomic(WB) ? (int64_t)ws.xscan[t] - b : 0;
    const int32_t sb = b + s * kLongSeg, se = min(sb + kLongSeg, e);
    for (int32_t k = sb + lane; k < se; k += 32)
        emit<T, WB>(ws, ym, __ldg(rowidx + k), S::mul(load_val(valc, k), xj), pos0 + k);
}

// Queues list entry t (column of `len` entries); returns false when the
// queue is full (the caller then walks the column itself).
// An entry reads (-1, 0) until its column is published, so a helper that
// sees the count before the entry skips it (its owner processes it).
__device__ __forceinline__ bool queue_long(const Ws& ws, int64_t t) {
    const unsigned q = atomicAdd(ws.lcol_n, 1u);
    if ((int32_t)q >= ws.lcol_cap) return false;
    *(volatile int32_t*)&ws.lcol[q].x = (int32_t)t;
    return true;
}

template <class T, int WB, bool WAIT>
__device__ __forceinline__ void help_long(const int32_t* __restrict__ colptr, const int32_t* __restrict__ rowidx,
                                          const T* __restrict__ valc, const CallDesc* __restrict__ desc,
                                          const Ws& ws, const uint32_t* ym, int lane, bool bm = false) {
    int32_t nq = 0;
    if (lane == 0) {
        const int64_t want = WAIT ? min(desc->nhub, (int64_t)ws.lcol_cap) : 0;
        nq = min((int32_t)*(volatile unsigned int*)ws.lcol_n, ws.lcol_cap);
        for (int it = 0; nq < want && it < kHubWaitIters; ++it) {
            __nanosleep(128);
            nq = min((int32_t)*(volatile unsigned int*)ws.lcol_n, ws.lcol_cap);
        }
    }
    nq = __shfl_sync(0xffffffffu, nq, 0);
    for (int32_t q = 0; q < nq; ++q) {
        int32_t t = 0, nseg = 0;
        if (lane == 0) {
            t = *(volatile int32_t*)&ws.lcol[q].x;
            for (int it = 0; WAIT && t < 0 && it < kHubWaitIters; ++it) {  // counted, not yet published
                __nanosleep(64);
                t = *(volatile int32_t*)&ws.lcol[q].x;
            }
            if (t >= 0) {
                const int32_t j = bm ? t : desc->xidx[t];
                nseg = (__ldg(colptr + j + 1) - __ldg(colptr + j) + kLongSeg - 1) / kLongSeg;
            }
        }
        t = __shfl_sync(0xffffffffu, t, 0);
        nseg = __shfl_sync(0xffffffffu, nseg, 0);
        if (t < 0) continue;  // not yet published: its owner will take it
        for (;;) {
            int32_t s = 0;
            if (lane == 0) s = atomicAdd(&ws.lcol[q].y, 1);
            s = __shfl_sync(0xffffffffu, s, 0);
            if (s >= nseg) break;
            push_segment<T, WB>(colptr, rowidx, valc, desc, ws, ym, t, s, lane, bm);
        }
    }
}

template <class T, int WB>
__global__ void __launch_bounds__(256) k_push_thread(const int32_t* __restrict__ colptr, const int32_t* __restrict__ rowidx,
                                                     const T* __restrict__ valc, const CallDesc* __restrict__ desc, Ws ws_in, Gate gate) {
    if (gate.off()) return;
    const Ws ws = push_ws<WB>(ws_in, desc);
    using S = Sr<T>;
    const uint32_t* __restrict__ ym = desc->ymask;
    const int lane = threadIdx.x & 31;
    const int64_t nx = desc->nnz_x;
    const int32_t* __restrict__ xidx = desc->xidx;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t tw = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); tw < nx; tw += stride) {
        const int64_t t = tw + lane;
        const bool valid = t < nx;
        T xj = S::one();
        int32_t b = 0, e = 0;
        int64_t pos0 = 0;
        if (valid) {
            const int32_t j = xidx[t];
            xj = list_val<T>(desc, t);
            b = __ldg(colptr + j);
            e = __ldg(colptr + j + 1);
            pos0 = !wb_atomic(WB) ? (int64_t)ws.xscan[t] - b : 0;
        }
        const bool lng = e - b > kLongCol;
        if (!lng) {
            // eight entries of the column loaded before their write-backs
            for (int32_t k0 = b; k0 < e; k0 += 8) {
                int32_t rr[8];
                typename S::Part pp[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    rr[u] = k0 + u < e ? __ldg(rowidx + k0 + u) : -1;
                    pp[u] = k0 + u < e ? S::mul(load_val(valc, k0 + u), xj) : typename S::Part(0);
                }
                emit_batch<T, WB, 8>(ws, ym, rr, pp, pos0 + k0, 1);
            }
        }
        // hubs go to the shared queue; the rest of the long columns to the warp
        const bool queued = lng && e - b > kLongSeg && queue_long(ws, t);
        for (unsigned pend = __ballot_sync(0xffffffffu, lng && !queued); pend; pend &= pend - 1) {
            const int src = __ffs(pend) - 1;
            const int32_t bb = __shfl_sync(0xffffffffu, b, src), ee = __shfl_sync(0xffffffffu, e, src);
            const int64_t p0 = __shfl_sync(0xffffffffu, pos0, src);
            T xx = S::one();
            if constexpr (!S::kPattern) xx = __shfl_sync(0xffffffffu, xj, src);
            for (int32_t k = bb + lane; k < ee; k += 32)
                emit<T, WB>(ws, ym, __ldg(rowidx + k), S::mul(load_val(valc, k), xx), p0 + k);
        }
    }
    // any lane may have queued a hub of this warp; lane 0 reads the queue
    // entries, so order those lanes' stores before its reads
    __syncwarp();
    help_long<T, WB, true>(colptr, rowidx, valc, desc, ws, ym, lane);
}

// One warp per listed column, G consecutive list entries per warp and round:
// on a list that gives every warp two groups of 32 or more, G = 32 -- lane l
// loads the pointers of the group's column l, then the warp walks the
// group's columns of at most 32 entries four at a time, lane l taking entry
// l of each, so such a column costs one load latency instead of the chain
// list entry -> column pointers -> entries (the stencil's products at x
// density 0.1: 468 -> 407 us listed, 427 -> 356 us dense); groups of 8 on a
// list ten times shorter measured slower (137 -> 144 us), so shorter lists
// keep G = 1. Longer columns follow one after another; hubs go to the queue.
// With bits_below > 0 (a dense x, atomic write-back) an x of fewer nonzeros
// than that -- the lists that would keep G = 1 -- is read from the feature
// pass's bitmap instead of a compacted list: lane l of a warp takes bitmap
// word l of the warp's stretch of 32 words and, round by round, the next set
// bit of it, so a round holds up to 32 columns walked as a group (their x
// values gathered from the dense x); the list's compaction is skipped.
template <class T, int WB>
__global__ void __launch_bounds__(256) k_push_warp(const int32_t* __restrict__ colptr, const int32_t* __restrict__ rowidx,
                                                   const T* __restrict__ valc, const CallDesc* __restrict__ desc, Ws ws_in, Gate gate,
                                                   int64_t ncols, int64_t bits_below) {
    if (gate.off()) return;
    const Ws ws = push_ws<WB>(ws_in, desc);
    using S = Sr<T>;
    using P = typename S::Part;
    constexpr unsigned FULL = 0xffffffffu;
    const uint32_t* __restrict__ ym = desc->ymask;
    const int lane = threadIdx.x & 31;
    const int64_t nx = desc->nnz_x;
    const int32_t* __restrict__ xidx = desc->xidx;
    const int64_t wpb = blockDim.x / 32;
    const int64_t nw = (int64_t)gridDim.x * wpb;
    const int G = nx >= 64 * nw ? 32 : 1;
    // columns of a group walked together (their loads in flight at once);
    // eight measured slower than four (the stencil's listed products at x
    // densities 0.1 and 0.01: 408 -> 456 and 141 -> 177 us, 32 -> 40 registers)
    constexpr int GU = 4;
    const bool bm = wb_atomic(WB) && nx < bits_below;
    // one round: lane l holds column j (list entry t) when valid
    auto round = [&](bool valid, int32_t j, int64_t t, T xj) {
        int32_t b = 0, len = 0, pos0 = 0;
        if (valid) {
            b = __ldg(colptr + j);
            len = __ldg(colptr + j + 1) - b;
            if (!wb_atomic(WB)) pos0 = ws.xscan[t] - b;
        }
        const bool queued = valid && len > kLongSeg && queue_long(ws, bm ? (int64_t)j : t);
        for (unsigned pend = __ballot_sync(FULL, valid && len <= 32); pend;) {
            int32_t rr[GU];
            P pp[GU];
            int32_t ps[GU];
#pragma unroll
            for (int u = 0; u < GU; ++u) {
                const bool has = pend != 0u;
                const int src = has ? __ffs(pend) - 1 : 0;
                pend &= pend - 1u;
                const int32_t bb = __shfl_sync(FULL, b, src);
                const int32_t ll = __shfl_sync(FULL, len, src);
                T xx = S::one();
                if constexpr (!S::kPattern) xx = __shfl_sync(FULL, xj, src);
                const int32_t p0 = !wb_atomic(WB) ? __shfl_sync(FULL, pos0, src) : 0;
                const int32_t k = bb + lane;
                const bool on = has && lane < ll;
                rr[u] = on ? __ldg(rowidx + k) : -1;
                pp[u] = on ? S::mul(load_val(valc, k), xx) : P(0);
                ps[u] = p0 + k;
            }
            emit_slots<T, WB, GU>(ws, ym, rr, pp, ps);
        }
        for (unsigned pend = __ballot_sync(FULL, valid && len > 32 && !queued); pend; pend &= pend - 1u) {
            const int src = __ffs(pend) - 1;
            const int32_t bb = __shfl_sync(FULL, b, src), ee = bb + __shfl_sync(FULL, len, src);
            T xx = S::one();
            if constexpr (!S::kPattern) xx = __shfl_sync(FULL, xj, src);
            const int64_t p0 = !wb_atomic(WB) ? (int64_t)__shfl_sync(FULL, pos0, src) : 0;
            for (int32_t k0 = bb + lane; k0 < ee; k0 += 128) {
                int32_t rr[4];
                P pp[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int32_t k = k0 + 32 * u;
                    rr[u] = k < ee ? __ldg(rowidx + k) : -1;
                    pp[u] = k < ee ? S::mul(load_val(valc, k), xx) : P(0);
                }
                emit_batch<T, WB, 4>(ws, ym, rr, pp, p0 + k0, 32);
            }
        }
    };
    const int64_t warp = blockIdx.x * wpb + (threadIdx.x >> 5);
    if (bm) {
        const uint32_t* __restrict__ xb = desc->xbits;
        const T* __restrict__ xd = (const T*)desc->x_dense;
        const int64_t nwords = (ncols + 31) >> 5;
        for (int64_t w0 = warp * 32; w0 < nwords; w0 += nw * 32) {
            uint32_t bits = w0 + lane < nwords ? __ldg(xb + w0 + lane) : 0u;
            while (__any_sync(FULL, bits != 0u)) {
                const bool valid = bits != 0u;
                const int32_t j = valid ? (int32_t)((w0 + lane) * 32 + __ffs(bits) - 1) : 0;
                bits &= bits - 1u;
                T xj = S::one();
                if constexpr (!S::kPattern) {
                    if (valid) xj = xd[j];
                }
                round(valid, j, 0, xj);
            }
        }
    } else {
        for (int64_t t0 = warp * G; t0 < nx; t0 += nw * G) {
            const int64_t t = t0 + lane;
            const bool valid = lane < G && t < nx;
            int32_t j = 0;
            T xj = S::one();
            if (valid) {
                j = xidx[t];
                xj = list_val<T>(desc, t);
            }
            round(valid, j, t, xj);
        }
    }
    // any lane may have queued a hub of this warp; lane 0 reads the queue
    // entries, so order those lanes' stores before its reads
    __syncwarp();
    help_long<T, WB, false>(colptr, rowidx, valc, desc, ws, ym, lane, bm);
}

// Even split: warp-chunks of 32*IPT effective nonzeros; the listed column of
// effective index e is the last t with xscan[t] <= e. A warp finds the range
// [t0, t1] of columns its chunk touches by two binary searches, then (when
// the range is short, the usual case) resolves every item's column with a
// load-balanced search in shared memory: each column's start is marked in a
// per-item table and a running maximum fills the gaps, while the columns'
// base offsets (colptr[j] - xscan[t]) and x values are staged beside it.
// Every item then costs one shared-memory read plus its own coalesced loads
// of the row index and value. Ranges longer than the chunk (runs of empty
// columns) fall back to one binary search per item.
template <class T, int WB>
__global__ void __launch_bounds__(256) k_push_bal(const int32_t* __restrict__ colptr, const int32_t* __restrict__ rowidx,
                                                  const T* __restrict__ valc, const CallDesc* __restrict__ desc, Ws ws_in, Gate gate) {
    if (gate.off()) return;
    const Ws ws = push_ws<WB>(ws_in, desc);
    using S = Sr<T>;
    constexpr int CH = 32 * kPushIPT;
    __shared__ int32_t s_t[8][CH];          // item -> list index of its column
    __shared__ int32_t s_base[8][CH + 1];   // column t0 + q: colptr[j] - xscan[t]
    __shared__ T s_xv[8][S::kPattern ? 1 : CH + 1];
    const uint32_t* __restrict__ ym = desc->ymask;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nx = desc->nnz_x, ns = desc->nnz_s;
    const int32_t* __restrict__ xidx = desc->xidx;
    const int32_t* __restrict__ sc = ws.xscan;
    const int64_t nchunks = (ns + CH - 1) / CH;
    const int64_t wpb = blockDim.x / 32;
    for (int64_t c = blockIdx.x * wpb + w; c < nchunks; c += (int64_t)gridDim.x * wpb) {
        const int64_t e0 = c * CH, elast = min(e0 + CH, ns) - 1;
        // the chunk's columns lie in [owner of e0, owner of the next chunk's
        // first item] (columns past elast start beyond the chunk and are skipped)
        const int64_t t0 = ws.chunk_t0[c];
        const int64_t t1 = (c + 1 < nchunks) ? (int64_t)ws.chunk_t0[c + 1] : nx - 1;
        const int nt = (int)(t1 - t0 + 1);
        if (nt <= CH + 1) {
            for (int i = lane; i < CH; i += 32) s_t[w][i] = -1;
            __syncwarp();
            for (int q = lane; q < nt; q += 32) {
                const int64_t t = t0 + q;
                const int32_t st = sc[t];
                s_base[w][q] = __ldg(colptr + xidx[t]) - st;
                if constexpr (!S::kPattern) s_xv[w][q] = list_val<T>(desc, t);
                const int64_t pos = max((int64_t)st - e0, (int64_t)0);
                if (pos < CH) atomicMax(&s_t[w][pos], (int32_t)q);
            }
            __syncwarp();
            // running maximum over the table: lane l owns entries 8l .. 8l+7
            int32_t run = -1;
            int32_t v[kPushIPT];
#pragma unroll
            for (int u = 0; u < kPushIPT; ++u) {
                run = max(run, s_t[w][lane * kPushIPT + u]);
                v[u] = run;
            }
            int32_t pre = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t other = __shfl_up_sync(0xffffffffu, pre, o);
                if (lane >= o) pre = max(pre, other);
            }
            int32_t carry = __shfl_up_sync(0xffffffffu, pre, 1);
            if (lane == 0) carry = -1;
            __syncwarp();
#pragma unroll
            for (int u = 0; u < kPushIPT; ++u) s_t[w][lane * kPushIPT + u] = max(v[u], carry);
            __syncwarp();
            // one write-back per item, four items per step: loading all eight
            // of a lane's items before the first write-back measured slower
            // (36 instead of 32 registers, six blocks per SM instead of eight:
            // 622 vs 588 us summed over one root's BFS levels of R-MAT scale 20)
#pragma unroll 4
            for (int s2 = 0; s2 < kPushIPT; ++s2) {
                const int64_t e = e0 + s2 * 32 + lane;
                if (e > elast) break;
                const int q = s_t[w][s2 * 32 + lane];
                const int64_t k = (int64_t)s_base[w][q] + e;
                const T xq = S::kPattern ? S::one() : s_xv[w][S::kPattern ? 0 : q];
                emit<T, WB>(ws, ym, __ldg(rowidx + k), S::mul(load_val(valc, k), xq), e);
            }
            __syncwarp();
        } else {
#pragma unroll 2
            for (int s2 = 0; s2 < kPushIPT; ++s2) {
                const int64_t e = e0 + s2 * 32 + lane;
                if (e > elast) break;
                int64_t lo = t0, hi = t1;
                while (lo < hi) {
                    const int64_t mid = (lo + hi + 1) >> 1;
                    if ((int64_t)sc[mid] <= e) lo = mid;
                    else hi = mid - 1;
                }
                const int32_t j = xidx[lo];
                const int64_t k = (int64_t)__ldg(colptr + j) + (e - sc[lo]);
                emit<T, WB>(ws, ym, __ldg(rowidx + k), S::mul(load_val(valc, k), list_val<T>(desc, lo)), e);
            }
        }
    }
}

// Exclusive scan of the listed columns' lengths, xscan[0..nnz_x], in two
// launches. Pass 1: each block writes its entries' lengths and their sum.
template <int B>
__global__ void __launch_bounds__(B) k_list_deg(const int32_t* __restrict__ colptr, const CallDesc* __restrict__ desc,
                                                int32_t* deg, int32_t* blk, Gate gate) {
    if (gate.off()) return;
    __shared__ int32_t sm[B / 32 + 1];
    const int64_t nx = desc->nnz_x;
    const int32_t* __restrict__ xidx = desc->xidx;
    int64_t lo, hi;
    block_range(nx, lo, hi);
    int32_t s = 0;
#pragma unroll 4
    for (int64_t t = lo + threadIdx.x; t < hi; t += B) {
        const int32_t j = __ldg(xidx + t);
        const int32_t d = __ldg(colptr + j + 1) - __ldg(colptr + j);
        deg[t] = d;
        s += d;
    }
    s = block_reduce_sum<B>(s, sm);
    if (threadIdx.x == 0) blk[blockIdx.x] = s;
}

// Pass 2: the lengths become their exclusive scan in place (runs of kRun per
// thread, one block scan per round, seeded with the sums of the blocks
// before). With OWNERS, entry t -- covering items [xscan[t], xscan[t] +
// len) -- also records itself as the owner of every balanced chunk whose
// first item it covers: each chunk start lies in exactly one non-empty
// entry, so no search and no atomics.
template <int B, bool OWNERS>
__global__ void __launch_bounds__(B) k_list_scan(int32_t* xscan, const CallDesc* __restrict__ desc,
                                                 const int32_t* __restrict__ blk, int32_t* chunk_t0, Gate gate) {
    if (gate.off()) return;
    constexpr int CH = 32 * kPushIPT;
    __shared__ int32_t sm[B / 32 + 1];
    const int64_t nx = desc->nnz_x;
    int64_t lo, hi;
    block_range(nx, lo, hi);
    int32_t base = block_prefix<B>(blk, blockIdx.x, sm);
    for (int64_t off = lo; off < hi; off += (int64_t)B * kRun) {
        const int64_t t0 = off + (int64_t)threadIdx.x * kRun;
        int32_t v[kRun];
#pragma unroll
        for (int q = 0; q < kRun; ++q) v[q] = t0 + q < hi ? xscan[t0 + q] : 0;
        int32_t c = 0;
#pragma unroll
        for (int q = 0; q < kRun; ++q) c += v[q];
        int32_t tot;
        int32_t e = base + block_excl_scan<B>(c, sm, &tot);
#pragma unroll
        for (int q = 0; q < kRun; ++q) {
            const bool valid = t0 + q < hi;
            if (valid) xscan[t0 + q] = e;
            if (OWNERS) {
                // chunks [c0, c1) start inside this entry's items; a hub
                // column's run of chunks is written by the whole warp
                const int64_t c0 = ((int64_t)e + CH - 1) / CH, c1 = ((int64_t)e + v[q] + CH - 1) / CH;
                const int64_t cnt = valid ? c1 - c0 : 0;
                if (cnt <= 8)
                    for (int64_t ch = c0; ch < c0 + cnt; ++ch) chunk_t0[ch] = (int32_t)(t0 + q);
                for (unsigned pend = __ballot_sync(0xffffffffu, cnt > 8); pend; pend &= pend - 1) {
                    const int src = __ffs(pend) - 1;
                    const int64_t lo = __shfl_sync(0xffffffffu, c0, src), n1 = __shfl_sync(0xffffffffu, c1, src);
                    const int32_t owner = (int32_t)__shfl_sync(0xffffffffu, t0 + q, src);
                    for (int64_t ch = lo + (threadIdx.x & 31); ch < n1; ch += 32) chunk_t0[ch] = owner;
                }
            }
            e += valid ? v[q] : 0;
        }
        base += tot;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) xscan[nx] = base;
}

// ---------------------------------------------------------------- sort write-back: reduce-by-key
// Warp-chunks of the row-sorted pairs: a segmented warp scan per round of 32
// pairs, a carry across the chunk's rounds, and one write per segment --
// a plain store for segments inside the chunk, an atomic add for the (at
// most two) segments that may be shared with a neighbouring chunk.
template <class T>
__global__ void __launch_bounds__(256) k_reduce_by_key(const uint32_t* __restrict__ keys, const T* __restrict__ vals,
                                                       const CallDesc* __restrict__ desc, Ws ws) {
    using S = Sr<T>;
    using P = typename S::Part;
    using A = typename S::Atom;
    constexpr int CH = 32 * kPushIPT;
    const int lane = threadIdx.x & 31;
    const int64_t ns = desc->nnz_s;
    const int64_t nchunks = (ns + CH - 1) / CH;
    const int64_t wpb = blockDim.x / 32;
    const uint32_t* __restrict__ ym = desc->ymask;
    A* acc = (A*)ws.acc;
    for (int64_t c = blockIdx.x * wpb + (threadIdx.x >> 5); c < nchunks; c += (int64_t)gridDim.x * wpb) {
        const int64_t e0 = c * CH, eend = min(e0 + CH, ns);
        const uint32_t first_key = keys[e0];
        uint32_t ckey = 0xffffffffu;
        P cval = P(0);
        for (int64_t r0 = e0; r0 < eend; r0 += 32) {
            const int64_t e = r0 + lane;
            const bool valid = e < eend;
            const uint32_t key = valid ? keys[e] : 0xffffffffu;
            // the segment carried from the previous round ended exactly at
            // the round boundary: write it out before this round starts
            if (r0 > e0 && __shfl_sync(0xffffffffu, key, 0) != ckey && lane == 0 && !row_masked(ym, ckey)) {
                if constexpr (!S::kPattern) {
                    if (ckey == first_key) atomicAdd(acc + ckey, S::to_atom(S::part_T(cval)));
                    else acc[ckey] = S::to_atom(S::part_T(cval));
                }
                ws.yflag[ckey] = 1;
            }
            P v = P(0);
            if constexpr (!S::kPattern) v = valid ? S::part_of(vals[e]) : P(0);
            else v = valid ? 1u : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const P pv = shfl_up(v, o);
                const uint32_t pk = shfl_up(key, o);
                if (lane >= o && pk == key) v = S::part_add(pv, v);
            }
            if (valid && key == ckey) v = S::part_add(cval, v);
            const uint32_t nk = __shfl_down_sync(0xffffffffu, key, 1);
            const bool last_lane = (lane == 31) || (r0 + lane + 1 >= eend);
            const bool seg_end = valid && (last_lane ? false : nk != key);
            if (seg_end && !row_masked(ym, key)) {
                if constexpr (!S::kPattern) {
                    if (key == first_key) atomicAdd(acc + key, S::to_atom(S::part_T(v)));
                    else acc[key] = S::to_atom(S::part_T(v));
                }
                ws.yflag[key] = 1;
            }
            // the segment running into the last valid lane carries on
            const int src = (int)min((int64_t)31, eend - 1 - r0);
            ckey = __shfl_sync(0xffffffffu, key, src);
            cval = __shfl_sync(0xffffffffu, v, src);
        }
        if (lane == 0 && !row_masked(ym, ckey)) {
            if constexpr (!S::kPattern) atomicAdd(acc + ckey, S::to_atom(S::part_T(cval)));
            ws.yflag[ckey] = 1;
        }
    }
}

// ---------------------------------------------------------------- privatised write-back
__global__ void k_bin_count(const uint32_t* __restrict__ keys, const CallDesc* __restrict__ desc, int32_t* bins,
                            int32_t nbins) {
    extern __shared__ int32_t sh[];
    const bool use_sm = nbins <= 8192;
    if (use_sm) {
        for (int i = threadIdx.x; i < nbins; i += blockDim.x) sh[i] = 0;
        __syncthreads();
    }
    const int64_t ns = desc->nnz_s;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ns; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t b = (int32_t)(keys[e] >> kPrivBits);
        if (use_sm) atomicAdd(&sh[b], 1);
        else atomicAdd(&bins[b], 1);
    }
    if (use_sm) {
        __syncthreads();
        for (int i = threadIdx.x; i < nbins; i += blockDim.x)
            if (sh[i]) atomicAdd(&bins[i], sh[i]);
    }
}

template <class T>
__global__ void k_bin_scatter(const uint32_t* __restrict__ kin, const T* __restrict__ vin, uint32_t* kout, T* vout,
                              const CallDesc* __restrict__ desc, int32_t* cursor) {
    const int64_t ns = desc->nnz_s;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ns; e += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = kin[e];
        const int32_t pos = atomicAdd(&cursor[k >> kPrivBits], 1);
        kout[pos] = k;
        if constexpr (!Sr<T>::kPattern) vout[pos] = vin[e];
    }
}

// One CTA per row tile: shared-memory accumulators (FP64 for the float types),
// then the tile's rows and bitmap words are written with plain stores.
template <class T>
__global__ void __launch_bounds__(256) k_priv_accumulate(const uint32_t* __restrict__ keys, const T* __restrict__ vals,
                                                         const int32_t* __restrict__ binoff, int64_t m, Ws ws,
                                                         const CallDesc* __restrict__ desc) {
    using S = Sr<T>;
    using A = typename S::Atom;
    constexpr int R = 1 << kPrivBits;
    __shared__ A s_acc[S::kPattern ? 1 : R];
    __shared__ uint32_t s_flag[R / 32];
    const int64_t tile = blockIdx.x;
    for (int i = threadIdx.x; i < R / 32; i += blockDim.x) s_flag[i] = 0u;
    if constexpr (!S::kPattern)
        for (int i = threadIdx.x; i < R; i += blockDim.x) s_acc[i] = A(0);
    __syncthreads();
    const int32_t b = binoff[tile], e = binoff[tile + 1];
    for (int32_t q = b + threadIdx.x; q < e; q += blockDim.x) {
        const int li = (int)(keys[q] & (R - 1));
        if constexpr (!S::kPattern) atomicAdd(&s_acc[li], S::to_atom(vals[q]));
        atomicOr(&s_flag[li >> 5], 1u << (li & 31));
    }
    __syncthreads();
    const int64_t row0 = tile * R;
    A* acc = (A*)ws.acc;
    for (int i = threadIdx.x; i < R; i += blockDim.x) {
        const int64_t r = row0 + i;
        if (r < m && ((s_flag[i >> 5] >> (i & 31)) & 1u) && !row_masked(desc->ymask, r)) {
            if constexpr (!S::kPattern) acc[r] = s_acc[i];
            ws.yflag[r] = 1;
        }
    }
}

// ---------------------------------------------------------------- launcher
static int bitlen64(int64_t v) {
    int b = 0;
    while (v > 0) { ++b; v >>= 1; }
    return b;
}

template <class T>
static void push_dtype(asv_matrix_s* H, int dist, int wb, int out_mode, cudaStream_t s, int64_t bits_below) {
    const T* valc = (const T*)H->val_csc;
    // a few blocks per SM for the per-column traversals (they stride over the
    // list, and a large grid of mostly idle blocks costs launch time on short
    // lists); more, smaller waves for the balanced one, whose chunks vary in cost
    const int grid = H->num_sms * 8;
    const CallDesc* d = H->d_desc;
    Ws ws = H->ws;
    const Gate gate = gate_of(H);
    // FP32 atomics where every row is short enough (see above) and the output
    // is dense, added straight into the zeroed output: no flags and no
    // write-out pass (FP32 accumulators written out by a pass took the
    // stencil's products at x densities 0.1 and 0.01 from 490 to 434 and from
    // 182 to 135 us against FP64 ones); the list output's compaction measured
    // slower on FP32 accumulators (94.9 -> 202.7 us for a 15.8M-row list) and
    // keeps FP64
    if (std::is_same<T, float>::value && wb == WB_ATOM && H->narrow_acc && out_mode == ASV_OUT_DENSE) wb = WB_ATOM_N;
    if (dist == 2 || !wb_atomic(wb)) {
        k_list_deg<256><<<H->G, 256, 0, s>>>(H->colptr, d, ws.xscan, ws.blk, gate);
        if (dist == 2)
            k_list_scan<256, true><<<H->G, 256, 0, s>>>(ws.xscan, d, ws.blk, ws.chunk_t0, gate);
        else
            k_list_scan<256, false><<<H->G, 256, 0, s>>>(ws.xscan, d, ws.blk, ws.chunk_t0, gate);
    }
#define TRAV(WBV)                                                                                   \
    do {                                                                                            \
        if (dist == 0) k_push_thread<T, WBV><<<grid, 256, 0, s>>>(H->colptr, H->rowidx, valc, d, ws, gate); \
        else if (dist == 1) k_push_warp<T, WBV><<<grid, 256, 0, s>>>(H->colptr, H->rowidx, valc, d, ws, gate, H->n, bits_below); \
        else k_push_bal<T, WBV><<<grid * 4, 256, 0, s>>>(H->colptr, H->rowidx, valc, d, ws, gate); \
    } while (0)
    if (wb == WB_ATOM_N) {
        if constexpr (std::is_same<T, float>::value) {
            if (H->m > 0) k_zero_out<T><<<H->num_sms * 4, 256, 0, s>>>(H->m, d, gate);
            TRAV(WB_ATOM_N);
        }
    } else if (wb == WB_ATOM) {
        TRAV(WB_ATOM);
    } else {
        TRAV(WB_SORT);
    }
#undef TRAV
    using V = PV<T>;
    if (wb == WB_SORT) {
        uint32_t* kb[2] = {ws.pkeys[0], ws.pkeys[1]};
        V* vb[2] = {(V*)ws.pvals[0], (V*)ws.pvals[1]};
        int cur;
        if (Sr<T>::kPattern)
            cur = radix_sort<V, false>(kb, vb, 0, &H->d_desc->nnz_s, bitlen64(H->m - 1), ws.hist, ws.blk, H->G, s);
        else
            cur = radix_sort<V, true>(kb, vb, 0, &H->d_desc->nnz_s, bitlen64(H->m - 1), ws.hist, ws.blk, H->G, s);
        k_reduce_by_key<T><<<grid, 256, 0, s>>>(kb[cur], (const T*)vb[cur], d, ws);
    } else if (wb == WB_PRIV) {
        const int32_t nbins = (int32_t)((H->m + (1 << kPrivBits) - 1) >> kPrivBits);
        int32_t* bins = ws.hist;  // nbins+1 counts, then offsets
        int32_t* cursor = ws.hist + (nbins + 1);
        cudaMemsetAsync(bins, 0, sizeof(int32_t) * (nbins + 1), s);
        const size_t shm = nbins <= 8192 ? sizeof(int32_t) * nbins : 0;
        k_bin_count<<<grid, 256, shm, s>>>(ws.pkeys[0], d, bins, nbins);
        scan_excl(bins, bins, nbins, nullptr, ws.blk, H->G, true, s);
        cudaMemcpyAsync(cursor, bins, sizeof(int32_t) * nbins, cudaMemcpyDeviceToDevice, s);
        k_bin_scatter<T><<<grid, 256, 0, s>>>(ws.pkeys[0], (const T*)ws.pvals[0], ws.pkeys[1], (T*)ws.pvals[1], d, cursor);
        if (nbins > 0) k_priv_accumulate<T><<<nbins, 256, 0, s>>>(ws.pkeys[1], (const T*)ws.pvals[1], bins, H->m, ws, d);
    }
    if (wb != WB_ATOM_N) launch_finalize(H, true, out_mode, s);
}

void launch_push(asv_matrix_s* H, int dist, int wb, int out_mode, cudaStream_t s, int64_t bits_below) {
    switch (H->dtype) {
        case ASV_F32: push_dtype<float>(H, dist, wb, out_mode, s, bits_below); break;
        case ASV_F64: push_dtype<double>(H, dist, wb, out_mode, s, bits_below); break;
        case ASV_I32: push_dtype<int32_t>(H, dist, wb, out_mode, s, bits_below); break;
        case ASV_BOOL: push_dtype<bool8>(H, dist, wb, out_mode, s, bits_below); break;
    }
}

int64_t priv_bins(int64_t m) { return (m + (1 << kPrivBits) - 1) >> kPrivBits; }

}  // namespace asv
