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
// result by more than one rounding.
#include "internal.h"
#include "prims.cuh"
#include "sort.cuh"

namespace asv {

enum { WB_ATOM = 0, WB_SORT = 1, WB_PRIV = 2 };
constexpr int kPrivBits = 12;  // rows per privatised tile = 4096
constexpr int kPushIPT = 8;    // effective nonzeros per lane per balanced chunk

template <class T>
using PV = typename std::conditional<sizeof(T) == 8, uint64_t, uint32_t>::type;

// One effective nonzero (row r, product p) at effective index pos.
template <class T, int WB>
__device__ __forceinline__ void emit(const Ws& ws, const uint32_t* ymask, int32_t r, typename Sr<T>::Part p,
                                     int64_t pos) {
    using S = Sr<T>;
    if (WB == WB_ATOM) {
        if (row_masked(ymask, r)) return;  // excluded by the output mask (pairs are masked when reduced)
        if constexpr (!S::kPattern) atomicAdd((typename S::Atom*)ws.acc + r, S::to_atom(S::part_T(p)));
        ws.yflag[r] = 1;
    } else {
        ws.pkeys[0][pos] = (uint32_t)r;
        if constexpr (!S::kPattern) {
            const T v = S::part_T(p);
            ((T*)ws.pvals[0])[pos] = v;
        }
    }
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

template <class T, int WB>
__global__ void __launch_bounds__(256) k_push_thread(const int32_t* __restrict__ colptr, const int32_t* __restrict__ rowidx,
                                                     const T* __restrict__ valc, const CallDesc* __restrict__ desc, Ws ws) {
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
            pos0 = (WB != WB_ATOM) ? (int64_t)ws.xscan[t] - b : 0;
        }
        const bool lng = e - b > kLongCol;
        if (!lng)
            for (int32_t k = b; k < e; ++k) emit<T, WB>(ws, ym, __ldg(rowidx + k), S::mul(load_val(valc, k), xj), pos0 + k);
        for (unsigned pend = __ballot_sync(0xffffffffu, lng); pend; pend &= pend - 1) {
            const int src = __ffs(pend) - 1;
            const int32_t bb = __shfl_sync(0xffffffffu, b, src), ee = __shfl_sync(0xffffffffu, e, src);
            const int64_t p0 = __shfl_sync(0xffffffffu, pos0, src);
            T xx = S::one();
            if constexpr (!S::kPattern) xx = __shfl_sync(0xffffffffu, xj, src);
            for (int32_t k = bb + lane; k < ee; k += 32)
                emit<T, WB>(ws, ym, __ldg(rowidx + k), S::mul(load_val(valc, k), xx), p0 + k);
        }
    }
}

template <class T, int WB>
__global__ void __launch_bounds__(256) k_push_warp(const int32_t* __restrict__ colptr, const int32_t* __restrict__ rowidx,
                                                   const T* __restrict__ valc, const CallDesc* __restrict__ desc, Ws ws) {
    using S = Sr<T>;
    const uint32_t* __restrict__ ym = desc->ymask;
    const int lane = threadIdx.x & 31;
    const int64_t nx = desc->nnz_x;
    const int32_t* __restrict__ xidx = desc->xidx;
    const int64_t wpb = blockDim.x / 32;
    for (int64_t t = blockIdx.x * wpb + (threadIdx.x >> 5); t < nx; t += (int64_t)gridDim.x * wpb) {
        const int32_t j = xidx[t];
        const T xj = list_val<T>(desc, t);
        const int32_t b = __ldg(colptr + j), e = __ldg(colptr + j + 1);
        const int64_t pos0 = (WB != WB_ATOM) ? (int64_t)ws.xscan[t] - b : 0;
        for (int32_t k = b + lane; k < e; k += 32) emit<T, WB>(ws, ym, __ldg(rowidx + k), S::mul(load_val(valc, k), xj), pos0 + k);
    }
}

// Even split: warp-chunks of 32*IPT effective nonzeros; the listed column of
// effective index e is the last t with xscan[t] <= e (binary search inside
// the chunk's column range).
template <class T, int WB>
__global__ void __launch_bounds__(256) k_push_bal(const int32_t* __restrict__ colptr, const int32_t* __restrict__ rowidx,
                                                  const T* __restrict__ valc, const CallDesc* __restrict__ desc, Ws ws) {
    using S = Sr<T>;
    const uint32_t* __restrict__ ym = desc->ymask;
    constexpr int CH = 32 * kPushIPT;
    const int lane = threadIdx.x & 31;
    const int64_t nx = desc->nnz_x, ns = desc->nnz_s;
    const int32_t* __restrict__ xidx = desc->xidx;
    const int32_t* __restrict__ sc = ws.xscan;
    const int64_t nchunks = (ns + CH - 1) / CH;
    const int64_t wpb = blockDim.x / 32;
    for (int64_t c = blockIdx.x * wpb + (threadIdx.x >> 5); c < nchunks; c += (int64_t)gridDim.x * wpb) {
        const int64_t e0 = c * CH, elast = min(e0 + CH, ns) - 1;
        int64_t bound = 0;
        if (lane < 2) {
            const int64_t target = lane == 0 ? e0 : elast;
            int64_t lo = 0, hi = nx - 1;
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if ((int64_t)sc[mid] <= target) lo = mid;
                else hi = mid - 1;
            }
            bound = lo;
        }
        const int64_t t0 = __shfl_sync(0xffffffffu, bound, 0), t1 = __shfl_sync(0xffffffffu, bound, 1);
#pragma unroll 2
        for (int s = 0; s < kPushIPT; ++s) {
            const int64_t e = e0 + s * 32 + lane;
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

// degree of each listed column, then an exclusive scan gives xscan[0..nnz_x]
__global__ void k_list_deg(const int32_t* __restrict__ colptr, const CallDesc* __restrict__ desc, int32_t* deg) {
    const int64_t nx = desc->nnz_x;
    const int32_t* xidx = desc->xidx;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nx; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j = xidx[t];
        deg[t] = __ldg(colptr + j + 1) - __ldg(colptr + j);
    }
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
static void push_dtype(asv_matrix_s* H, int dist, int wb, int out_mode, cudaStream_t s) {
    const T* valc = (const T*)H->val_csc;
    const int grid = H->num_sms * 32;
    const CallDesc* d = H->d_desc;
    Ws ws = H->ws;
    if (dist == 2 || wb != WB_ATOM) {
        k_list_deg<<<grid, 256, 0, s>>>(H->colptr, d, ws.xscan);
        scan_excl(ws.xscan, ws.xscan, 0, &H->d_desc->nnz_x, ws.blk, H->G, true, s);
    }
#define TRAV(WBV)                                                                                   \
    do {                                                                                            \
        if (dist == 0) k_push_thread<T, WBV><<<grid, 256, 0, s>>>(H->colptr, H->rowidx, valc, d, ws); \
        else if (dist == 1) k_push_warp<T, WBV><<<grid, 256, 0, s>>>(H->colptr, H->rowidx, valc, d, ws); \
        else k_push_bal<T, WBV><<<grid, 256, 0, s>>>(H->colptr, H->rowidx, valc, d, ws);          \
    } while (0)
    if (wb == WB_ATOM) TRAV(WB_ATOM);
    else TRAV(WB_SORT);
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
    launch_finalize(H, true, out_mode, s);
}

void launch_push(asv_matrix_s* H, int dist, int wb, int out_mode, cudaStream_t s) {
    switch (H->dtype) {
        case ASV_F32: push_dtype<float>(H, dist, wb, out_mode, s); break;
        case ASV_F64: push_dtype<double>(H, dist, wb, out_mode, s); break;
        case ASV_I32: push_dtype<int32_t>(H, dist, wb, out_mode, s); break;
        case ASV_BOOL: push_dtype<bool8>(H, dist, wb, out_mode, s); break;
    }
}

int64_t priv_bins(int64_t m) { return (m + (1 << kPrivBits) - 1) >> kPrivBits; }

}  // namespace asv
