// Parallel primitives used by the runtime procedure (Sec. VI-C: "reduction,
// prefix sum and stream compaction") and by the sort-based write-back
// (Sec. IV-B): block/device exclusive scans, a stable LSD radix sort of
// 32-bit keys with optional payload, and ordered bitmap compaction.
#pragma once
#include "common.cuh"

namespace asv {

// ---------------------------------------------------------------- block helpers
template <int B, class V>
__device__ __forceinline__ V block_reduce_sum(V v, V* sm /* >= B/32 */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    if (lane == 0) sm[wid] = v;
    __syncthreads();
    V r = 0;
    if (wid == 0) {
        r = (lane < B / 32) ? sm[lane] : V(0);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) r += __shfl_xor_sync(0xffffffffu, r, d);
        if (lane == 0) sm[0] = r;
    }
    __syncthreads();
    r = sm[0];
    __syncthreads();
    return r;
}

// Exclusive block scan of one value per thread; *total receives the sum.
template <int B, class V>
__device__ __forceinline__ V block_excl_scan(V v, V* sm /* >= B/32 + 1 */, V* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    V inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        V o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) sm[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        V w = (lane < B / 32) ? sm[lane] : V(0);
        V wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            V o = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += o;
        }
        if (lane < B / 32) sm[lane] = wi - w;  // exclusive warp offsets
        if (lane == B / 32 - 1) sm[B / 32] = wi;
    }
    __syncthreads();
    V r = sm[wid] + inc - v;
    if (total) *total = sm[B / 32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ int64_t dev_count(int64_t host_n, const int64_t* dev_n) {
    return dev_n ? *dev_n : host_n;
}

// ---------------------------------------------------------------- device exclusive scan
// Items per thread and round in the second pass of a scan or compaction: a
// thread loads a contiguous run (independent loads, one memory latency) and
// the block scans the runs' totals once per B * kRun items.
constexpr int kRun = 8;

// Block b of the grid owns [lo, hi); the chunk is a whole number of runs, so
// runs start 32-byte aligned relative to the array and never straddle blocks.
__device__ __forceinline__ void block_range(int64_t n, int64_t& lo, int64_t& hi) {
    int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    chunk = (chunk + kRun - 1) / kRun * kRun;
    lo = min(n, (int64_t)blockIdx.x * chunk);
    hi = min(n, lo + chunk);
}

// Two launches over a fixed grid of G blocks, each owning one contiguous
// range: per-block sums, then per-block scans seeded with the block's offset
// (the sum of the block sums before it). Deterministic; n may live on the
// device.
template <int B>
__global__ void __launch_bounds__(B) k_scan_reduce(const int32_t* in, int64_t n_h, const int64_t* n_d,
                                                   int32_t* blk) {
    __shared__ int32_t sm[B / 32 + 1];
    const int64_t n = dev_count(n_h, n_d);
    int64_t lo, hi;
    block_range(n, lo, hi);
    int32_t s = 0;
#pragma unroll 4
    for (int64_t i = lo + threadIdx.x; i < hi; i += B) s += in[i];
    s = block_reduce_sum<B>(s, sm);
    if (threadIdx.x == 0) blk[blockIdx.x] = s;
}

// Sum of blk[0 .. b) by the whole block: each block of a scan or compaction
// finds its own offset among the G (a few hundred) block totals, which saves
// a separate one-block scan launch between the two passes.
template <int B>
__device__ __forceinline__ int32_t block_prefix(const int32_t* __restrict__ blk, int b, int32_t* sm /* >= B/32+1 */) {
    int32_t s = 0;
    for (int i = threadIdx.x; i < b; i += B) s += blk[i];
    return block_reduce_sum<B>(s, sm);
}

template <int B>
__global__ void __launch_bounds__(B) k_scan_down(const int32_t* in, int32_t* out, int64_t n_h,
                                                 const int64_t* n_d, const int32_t* blk, int write_total) {
    __shared__ int32_t sm[B / 32 + 1];
    const int64_t n = dev_count(n_h, n_d);
    int64_t lo, hi;
    block_range(n, lo, hi);
    const bool vec = (((uintptr_t)in | (uintptr_t)out) & 15) == 0;
    int32_t base = block_prefix<B>(blk, blockIdx.x, sm);  // blk holds the raw block sums
    for (int64_t off = lo; off < hi; off += (int64_t)B * kRun) {
        const int64_t i0 = off + (int64_t)threadIdx.x * kRun;
        const bool full = vec && i0 + kRun <= hi;
        int32_t v[kRun];
        if (full) {
            const int4 a = *reinterpret_cast<const int4*>(in + i0);
            const int4 b = *reinterpret_cast<const int4*>(in + i0 + 4);
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
            v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        } else {
#pragma unroll
            for (int q = 0; q < kRun; ++q) v[q] = i0 + q < hi ? in[i0 + q] : 0;
        }
        int32_t c = 0;
#pragma unroll
        for (int q = 0; q < kRun; ++q) c += v[q];
        int32_t tot;
        int32_t e = base + block_excl_scan<B>(c, sm, &tot);
#pragma unroll
        for (int q = 0; q < kRun; ++q) {
            const int32_t x = v[q];
            v[q] = e;
            e += x;
        }
        if (full) {
            *reinterpret_cast<int4*>(out + i0) = make_int4(v[0], v[1], v[2], v[3]);
            *reinterpret_cast<int4*>(out + i0 + 4) = make_int4(v[4], v[5], v[6], v[7]);
        } else {
#pragma unroll
            for (int q = 0; q < kRun; ++q)
                if (i0 + q < hi) out[i0 + q] = v[q];
        }
        base += tot;
    }
    if (write_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = base;
}

// ---------------------------------------------------------------- radix sort (LSD, 8-bit digits)
template <int B>
__global__ void __launch_bounds__(B) k_radix_hist(const uint32_t* keys, int64_t n_h, const int64_t* n_d,
                                                  int shift, int32_t* hist /* [256][G] */) {
    __shared__ int32_t h[256];
    for (int d = threadIdx.x; d < 256; d += B) h[d] = 0;
    __syncthreads();
    const int64_t n = dev_count(n_h, n_d);
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * chunk, hi = min(n, lo + chunk);
    for (int64_t i = lo + threadIdx.x; i < hi; i += B) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += B) hist[(int64_t)d * gridDim.x + blockIdx.x] = h[d];
}

// Stable scatter: items of a block keep their order within each digit
// (warp match + per-warp digit counts per round of B items), and blocks are
// ordered by the digit-major exclusive scan of the histogram.
template <int B, class V, bool HAS_V>
__global__ void __launch_bounds__(B) k_radix_scatter(const uint32_t* kin, const V* vin, uint32_t* kout,
                                                     V* vout, int64_t n_h, const int64_t* n_d, int shift,
                                                     const int32_t* offs /* [256][G] exclusive */) {
    constexpr int NW = B / 32;
    __shared__ int32_t base[256];
    __shared__ int32_t cnt[NW][257];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < 256; d += B) base[d] = offs[(int64_t)d * gridDim.x + blockIdx.x];
    const int64_t n = dev_count(n_h, n_d);
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * chunk, hi = min(n, lo + chunk);
    for (int64_t off = lo; off < hi; off += B) {
        for (int e = threadIdx.x; e < NW * 257; e += B) (&cnt[0][0])[e] = 0;
        __syncthreads();
        const int64_t i = off + threadIdx.x;
        const bool valid = i < hi;
        uint32_t key = valid ? kin[i] : 0u;
        V v{};
        if (HAS_V && valid) v = vin[i];
        const int d = valid ? (int)((key >> shift) & 255u) : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lanemask_lt());
        if (rank == 0) cnt[wid][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int32_t pos = base[d] + rank;
            for (int w = 0; w < wid; ++w) pos += cnt[w][d];
            kout[pos] = key;
            if (HAS_V) vout[pos] = v;
        }
        __syncthreads();
        for (int dd = threadIdx.x; dd < 256; dd += B) {
            int32_t s = 0;
            for (int w = 0; w < NW; ++w) s += cnt[w][dd];
            base[dd] += s;
        }
        __syncthreads();
    }
}

}  // namespace asv
