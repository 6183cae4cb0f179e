// The (sub-)warp row-major kernel: its template and launcher, instantiated
// per value type in pull_warp_fp.cu and pull_warp_int.cu.
#pragma once
#include "pull_common.cuh"

namespace asv {

// ---------------------------------------------------------------- L lanes per row
// A group of L lanes owns one row; a warp owns RW = (32/L)*U consecutive rows,
// whose row pointers it reads with one coalesced load. Lane l reads its
// row's 16-byte-aligned 4-element chunks l, l+L, ... with one 128-bit load of
// column ids and one of values each (elements outside the row are masked).
// The first chunk of all U rows of a group is loaded before any x gather, so
// a warp keeps U*32 bytes per lane in flight. Chunk products are added as a
// small tree, chunks of a lane with compensated summation, and the group's
// lanes with shuffles.
template <class T, bool MASK, bool VEC>
struct Chunk {
    int32_t c[4];
    T v[4];
    bool in[4];
};

template <class T, bool MASK, bool VEC>
__device__ __forceinline__ void chunk_load(Chunk<T, MASK, VEC>& ch, const int32_t* __restrict__ col,
                                           const T* __restrict__ val, int64_t nnz, int32_t base, int32_t b, int32_t e) {
    using S = Sr<T>;
    const bool full = VEC && base < e && (int64_t)base + 4 <= nnz;
#pragma unroll
    for (int q = 0; q < 4; ++q) ch.in[q] = base + q >= b && base + q < e;
    if (full) {
        const int4 cc = __ldg(reinterpret_cast<const int4*>(col + base));
        ch.c[0] = cc.x; ch.c[1] = cc.y; ch.c[2] = cc.z; ch.c[3] = cc.w;
        if constexpr (!S::kPattern && !MASK) {
            if (val != nullptr) {
                if constexpr (sizeof(T) == 4) {
                    const int4 vv = __ldg(reinterpret_cast<const int4*>(val + base));
                    ch.v[0] = __int_as_float_t<T>(vv.x); ch.v[1] = __int_as_float_t<T>(vv.y);
                    ch.v[2] = __int_as_float_t<T>(vv.z); ch.v[3] = __int_as_float_t<T>(vv.w);
                } else {
                    const double2 v01 = __ldg(reinterpret_cast<const double2*>(val + base));
                    const double2 v23 = __ldg(reinterpret_cast<const double2*>(val + base + 2));
                    ch.v[0] = (T)v01.x; ch.v[1] = (T)v01.y; ch.v[2] = (T)v23.x; ch.v[3] = (T)v23.y;
                }
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) ch.v[q] = S::one();
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            ch.c[q] = ch.in[q] ? __ldg(col + base + q) : 0;
            if constexpr (!S::kPattern && !MASK) ch.v[q] = ch.in[q] ? load_val(val, base + q) : T(0);
        }
    }
    // a pattern chunk marks entries outside the row with column -1 (column
    // ids are non-negative), so it carries no separate in-range flags
    if constexpr (S::kPattern) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (!ch.in[q]) ch.c[q] = -1;
    }
}

template <class T, bool MASK, bool SOUT, bool VEC>
__device__ __forceinline__ typename Sr<T>::Part chunk_sum(Chunk<T, MASK, VEC>& ch, const T* __restrict__ val,
                                                          const T* __restrict__ x, const uint32_t* __restrict__ xbits,
                                                          int32_t base, bool& hit) {
    using S = Sr<T>;
    using P = typename S::Part;
    if constexpr (S::kPattern) {
        uint32_t any = 0u;
#pragma unroll
        for (int q = 0; q < 4; ++q) any |= ch.c[q] >= 0 ? bool_gather(x, xbits, ch.c[q]) : 0u;
        if (SOUT) hit |= any != 0u;
        return any;
    }
    bool eff[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        bool bit = true;
        if (MASK || SOUT) bit = ch.in[q] && test_bit(xbits, ch.c[q]);
        if (SOUT) hit |= bit;
        eff[q] = ch.in[q] && (!MASK || bit);
    }
    if constexpr (S::kPattern) {
#pragma unroll
        for (int q = 0; q < 4; ++q) ch.v[q] = S::one();
    } else if constexpr (MASK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) ch.v[q] = eff[q] ? load_val(val, base + q) : T(0);
    }
    P pr[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) pr[q] = eff[q] ? S::mul(ch.v[q], __ldg(x + ch.c[q])) : P(0);
    return S::part_add(S::part_add(pr[0], pr[1]), S::part_add(pr[2], pr[3]));
}

template <int L, int UU>
struct WarpRows {
    static constexpr int U = (L == 2 && UU > 2) ? 2 : UU;  // rows per group, loaded together
    static constexpr int RW = (32 / L) * U;                 // rows per warp (<= 32)
};

template <class T, bool MASK, bool SOUT, int L, bool VEC, int UU>
__global__ void __launch_bounds__(256, UU >= 4 ? 4 : 6) k_pull_warp(int64_t m, int64_t nnz, const int32_t* __restrict__ rowptr,
                                                   const int32_t* __restrict__ col, const T* __restrict__ val,
                                                   PullArg a, void* ywork, uint8_t* yflag) {
    using S = Sr<T>;
    using P = typename S::Part;
    constexpr int U = WarpRows<L, UU>::U, RW = WarpRows<L, UU>::RW, RPW = 32 / L;
    const PullIO p = resolve(a, ywork, SOUT);
    const T* __restrict__ x = (const T*)p.x;
    T* __restrict__ y = (T*)p.y;
    const int lane = threadIdx.x & 31, g = lane / L, l = lane % L;
    const int64_t row0 = ((int64_t)blockIdx.x * 8 + (threadIdx.x >> 5)) * RW;
    if (row0 >= m) return;
    const int32_t rp = (lane < RW && row0 + lane <= m) ? __ldg(rowptr + row0 + lane) : 0;
    const int32_t rp_end = __ldg(rowptr + min(row0 + RW, m));
    int32_t b[U], e[U];
    bool valid[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int r = u * RPW + g;
        valid[u] = row0 + r < m;
        b[u] = __shfl_sync(0xffffffffu, rp, r);
        const int32_t nx = __shfl_sync(0xffffffffu, rp, (r + 1) & 31);
        e[u] = (r + 1 == RW) ? rp_end : nx;
        if (e[u] - b[u] > kLongRow) valid[u] = false;  // summed by k_pull_long
        if (!valid[u] || row_masked(p.ymask, row0 + r)) e[u] = b[u];  // masked rows: y = 0
    }
    Chunk<T, MASK, VEC> ch[U];
#pragma unroll
    for (int u = 0; u < U; ++u) chunk_load(ch[u], col, val, nnz, (b[u] & ~3) + 4 * l, b[u], e[u]);
    P vs[U];
    bool hit[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        hit[u] = false;
        typename S::Acc acc;
        S::acc_zero(acc);
        const int32_t base0 = (b[u] & ~3) + 4 * l;
        S::acc_add(acc, chunk_sum<T, MASK, SOUT, VEC>(ch[u], val, x, p.xbits, base0, hit[u]));
        for (int32_t base = base0 + 4 * L; base < e[u]; base += 4 * L) {
            if constexpr (S::kPattern) {
                if (acc) break;  // OR is settled by the first hit
            }
            Chunk<T, MASK, VEC> c2;
            chunk_load(c2, col, val, nnz, base, b[u], e[u]);
            S::acc_add(acc, chunk_sum<T, MASK, SOUT, VEC>(c2, val, x, p.xbits, base, hit[u]));
        }
        vs[u] = S::acc_part(acc);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        P v = vs[u];
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) v = S::part_add(v, shfl_xor(v, o, L));
        bool h = false;
        if (SOUT) {
            const unsigned bal = __ballot_sync(0xffffffffu, hit[u]);
            const unsigned gm = (0xffffffffu >> (32 - L)) << (lane & ~(L - 1));
            h = (bal & gm) != 0;
        }
        if (valid[u] && l == 0) {
            const int64_t i = row0 + u * RPW + g;
            if (!(S::kPattern && SOUT)) y[i] = S::part_T(v);  // a Boolean sparse output is its flags
            if (SOUT && h) yflag[i] = 1;
        }
    }
}


// ---------------------------------------------------------------- long rows
// One warp per segment of a long row (at most kLongSeg entries, from a
// 16-byte descriptor built once per matrix): lane l reads
// 16-byte chunks l, l+32, ... of the segment with 128-bit loads, the next
// chunk's loads issued before the current chunk's gathers. Boolean segments
// stop as soon as any lane has a hit; for a Boolean sparse output a segment
// with a hit sets its row's flag and nothing else. Otherwise a row that is
// one segment is written directly, and the segments of a longer row leave
// their partials in part[] in the push-side accumulator type (FP64 for FP32
// values) for k_pull_long_fixup to add in segment order.
template <class A>
__device__ __forceinline__ uint64_t atom_bits(A v) {
    if constexpr (sizeof(A) == 8) return (uint64_t)__double_as_longlong(v);
    else return (uint64_t)v;
}

template <class A>
__device__ __forceinline__ A atom_from_bits(uint64_t b) {
    if constexpr (sizeof(A) == 8) return __longlong_as_double((long long)b);
    else return (A)b;
}

template <class T>
__device__ __forceinline__ typename Sr<T>::Atom atom_combine(typename Sr<T>::Atom a, typename Sr<T>::Atom b) {
    if constexpr (Sr<T>::kPattern) return a | b;
    else if constexpr (sizeof(typename Sr<T>::Atom) == 8) return __dadd_rn(a, b);
    else return a + b;
}

// Boolean products with a list output (BFS levels) hand the rest of a
// segment without a true term in its first kLongFirst chunks to a second
// pass: most segments stop within their first chunk, and the launch used to
// wait on the few that walked 32 chunks one load latency after another. The
// rest goes out as pieces of kLongPiece entries ({row, begin, end, 0}) that
// any warp of k_pull_long_rest takes.
constexpr int kLongFirst = 1;
constexpr int kLongPiece = 512;

// One warp's segment sg of a Boolean list-output product: its first
// kLongFirst chunks; a true term sets the row's flag, otherwise the rest of
// the segment is queued for k_pull_long_rest as pieces of kLongPiece entries.
template <bool MASK, bool VEC>
__device__ __forceinline__ void long_seg_bool_first(int64_t sg, int64_t nnz, const int4* __restrict__ seg,
                                                    const int32_t* __restrict__ col, const PullIO& p, uint8_t* yflag,
                                                    int4* rest, unsigned int* rest_n, int lane) {
    using T = bool8;
    const bool8* __restrict__ x = (const bool8*)p.x;
    const int4 d = __ldg(seg + sg);  // {row, begin, end, whole row}
    const int32_t row = d.x, b = d.y;
    const int32_t e = row_masked(p.ymask, row) ? b : d.z;  // a masked row has no term
    const int32_t a0 = b & ~3;
    const int nsteps = (e - a0 + 127) >> 7;
    const int lim = min(nsteps, kLongFirst);
    bool hit = false;
    uint32_t acc = 0u;
    Chunk<T, MASK, VEC> cur;
    chunk_load(cur, col, (const T*)nullptr, nnz, a0 + 4 * lane, b, e);
    for (int t = 0; t < lim; ++t) {
        const int32_t base = a0 + 128 * t + 4 * lane;
        Chunk<T, MASK, VEC> nxt;
        // the next chunk is loaded before this one's gathers -- unless this
        // is the last chunk this warp walks (the rest goes to the second pass)
        if (t + 1 < lim || lim == nsteps) chunk_load(nxt, col, (const T*)nullptr, nnz, base + 128, b, e);
        acc |= chunk_sum<T, MASK, true, VEC>(cur, (const T*)nullptr, x, p.xbits, base, hit);
        if (__any_sync(0xffffffffu, acc != 0u)) break;
        cur = nxt;
    }
    if (__any_sync(0xffffffffu, hit)) {
        if (lane == 0) yflag[row] = 1;
    } else if (lim < nsteps) {
        const int32_t r0 = a0 + 128 * lim;
        const int32_t np = (e - r0 + kLongPiece - 1) / kLongPiece;
        unsigned int q0 = 0;
        if (lane == 0) q0 = atomicAdd(rest_n, (unsigned int)np);
        q0 = __shfl_sync(0xffffffffu, q0, 0);
        for (int32_t k = lane; k < np; k += 32)
            rest[q0 + k] = make_int4(row, r0 + k * kLongPiece, min(e, r0 + (k + 1) * kLongPiece), 0);
    }
}

template <class T, bool MASK, bool SOUT, bool VEC>
__global__ void __launch_bounds__(256) k_pull_long(int64_t nseg, int64_t nnz, const int4* __restrict__ seg,
                                                   const int32_t* __restrict__ col, const T* __restrict__ val,
                                                   PullArg a, void* ywork, uint8_t* yflag, uint64_t* part,
                                                   uint8_t* part_hit, int4* rest, unsigned int* rest_n) {
    using S = Sr<T>;
    using P = typename S::Part;
    const PullIO p = resolve(a, ywork, SOUT);
    const T* __restrict__ x = (const T*)p.x;
    T* __restrict__ y = (T*)p.y;
    const int lane = threadIdx.x & 31;
    const int64_t sg = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (sg >= nseg) return;
    if constexpr (S::kPattern && SOUT) {
        if (rest != nullptr) {
            long_seg_bool_first<MASK, VEC>(sg, nnz, seg, col, p, yflag, rest, rest_n, lane);
            return;
        }
    }
    const int4 d = __ldg(seg + sg);  // {row, begin, end, whole row}
    const int32_t row = d.x, b = d.y;
    const int32_t e = row_masked(p.ymask, row) ? b : d.z;  // a masked row sums nothing (y = 0)
    const int32_t a0 = b & ~3;
    const int nsteps = (e - a0 + 127) >> 7;
    bool hit = false;
    typename S::Acc acc;
    S::acc_zero(acc);
    Chunk<T, MASK, VEC> cur;
    chunk_load(cur, col, val, nnz, a0 + 4 * lane, b, e);
    for (int t = 0; t < nsteps; ++t) {
        const int32_t base = a0 + 128 * t + 4 * lane;
        Chunk<T, MASK, VEC> nxt;
        chunk_load(nxt, col, val, nnz, base + 128, b, e);  // the next chunk before this one's gathers
        S::acc_add(acc, chunk_sum<T, MASK, SOUT, VEC>(cur, val, x, p.xbits, base, hit));
        if constexpr (S::kPattern) {
            // OR is settled by the first hit (a deeper prefetch, and warps
            // that keep the next segment's first chunk in flight, measured
            // slower: most long rows of a BFS level stop within their first
            // chunks)
            if (__any_sync(0xffffffffu, acc != 0u)) break;
        }
        cur = nxt;
    }
    P v = S::acc_part(acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = S::part_add(v, shfl_xor(v, o));
    const bool h = SOUT && __any_sync(0xffffffffu, hit);
    if constexpr (S::kPattern && SOUT) {
        // a Boolean sparse output is its flags: any segment with a true term
        // settles its row, so no partials and no fix-up
        if (h && lane == 0) yflag[row] = 1;
        return;
    }
    if (lane != 0) return;
    if (d.w) {
        y[row] = S::part_T(v);
        if (SOUT && h) yflag[row] = 1;
    } else {
        part[sg] = atom_bits(S::to_atom(v));
        if (SOUT) part_hit[sg] = h ? 1 : 0;
    }
}

// The second pass of the Boolean list-output products: a warp per piece,
// skipped when the row is already settled, stopping at the first true term.
template <class T, bool MASK, bool VEC>
__global__ void __launch_bounds__(256) k_pull_long_rest(const int4* __restrict__ rest,
                                                        const unsigned int* __restrict__ rest_n, int64_t nnz,
                                                        const int32_t* __restrict__ col, PullArg a, void* ywork,
                                                        uint8_t* yflag) {
    using S = Sr<T>;
    const PullIO p = resolve(a, ywork, true);
    const T* __restrict__ x = (const T*)p.x;
    const int lane = threadIdx.x & 31;
    const int64_t n = *rest_n;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < n; w += warps) {
        const int4 d = rest[w];
        int done = 0;
        if (lane == 0) done = *(volatile const uint8_t*)(yflag + d.x);
        if (__shfl_sync(0xffffffffu, done, 0)) continue;  // settled by another piece or the first chunks
        const int32_t b = d.y, e = d.z;
        const int nsteps = (e - b + 127) >> 7;
        bool hit = false;
        Chunk<T, MASK, VEC> cur;
        chunk_load(cur, col, (const T*)nullptr, nnz, b + 4 * lane, b, e);
        for (int t = 0; t < nsteps; ++t) {
            const int32_t base = b + 128 * t + 4 * lane;
            Chunk<T, MASK, VEC> nxt;
            chunk_load(nxt, col, (const T*)nullptr, nnz, base + 128, b, e);
            const typename S::Acc acc = chunk_sum<T, MASK, true, VEC>(cur, (const T*)nullptr, x, p.xbits, base, hit);
            if (__any_sync(0xffffffffu, acc != 0u)) {
                hit = true;
                break;
            }
            cur = nxt;
        }
        if (lane == 0 && hit) yflag[d.x] = 1;
    }
}

// Boolean products with a list output on a matrix with long rows (the BFS
// levels of a power-law graph): the long-row segments' first chunks and the
// one-row-per-thread walk of the other rows in one launch of 128-thread
// blocks. Blocks [0, lblocks) take four segments each (a warp per segment),
// the others 128 * kBoolRows rows each. Blocks are dispatched in about
// index order, so the segments -- whose first chunks and queued rests are
// the long pole -- start first and the row blocks fill the SMs as segment
// blocks finish, with no gap between two launches and no second stream.
template <bool MASK, bool VEC>
__global__ void __launch_bounds__(128) k_pull_bool_fused(int64_t m, int64_t nseg, int64_t nnz, unsigned lblocks,
                                                         const int32_t* __restrict__ rowptr,
                                                         const int4* __restrict__ seg, const int32_t* __restrict__ col,
                                                         PullArg a, void* ywork, uint8_t* yflag, int4* rest,
                                                         unsigned int* rest_n) {
    const PullIO p = resolve(a, ywork, true);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (blockIdx.x < lblocks) {
        const int64_t sg = (int64_t)blockIdx.x * 4 + w;
        if (sg < nseg) long_seg_bool_first<MASK, VEC>(sg, nnz, seg, col, p, yflag, rest, rest_n, lane);
        return;
    }
    const int64_t r0 = ((int64_t)(blockIdx.x - lblocks) * 4 + w) * 32 * kBoolRows;
    if (r0 >= m) return;
    pull_rows_bool<true>(m, rowptr, col, p, nullptr, yflag, r0, lane);
}

// The fused launch above, then the second pass over the queued rests (the
// Boolean list-output thread pull on a matrix with long rows).
void launch_pull_bool_fused(asv_matrix_s* H, const PullArg& a, bool masked, bool vec, cudaStream_t s);

template <class T>
__global__ void k_pull_long_fixup(int64_t nmulti, const int32_t* __restrict__ multi_row,
                                  const int32_t* __restrict__ multi_base, const int32_t* __restrict__ rowptr,
                                  const uint64_t* __restrict__ part, const uint8_t* __restrict__ part_hit, PullArg a,
                                  void* ywork, uint8_t* yflag, int sout) {
    using S = Sr<T>;
    using Atom = typename S::Atom;
    const PullIO p = resolve(a, ywork, sout != 0);
    T* __restrict__ y = (T*)p.y;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nmulti; q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t row = multi_row[q], base = multi_base[q];
        const int32_t k = (rowptr[row + 1] - rowptr[row] + kLongSeg - 1) / kLongSeg;
        Atom sum = atom_from_bits<Atom>(part[base]);
        bool h = sout && part_hit[base];
        for (int32_t t = 1; t < k; ++t) {
            sum = atom_combine<T>(sum, atom_from_bits<Atom>(part[base + t]));
            if (sout) h |= part_hit[base + t] != 0;
        }
        y[row] = S::from_atom(sum);
        if (sout && h) yflag[row] = 1;
    }
}

template <class T, bool MASK, bool SOUT>
void launch_pull_long_dtype(asv_matrix_s* H, const PullArg& a, bool vec, cudaStream_t s) {
    if (H->nseg == 0) return;
    const T* val = (const T*)H->val;
    const unsigned g = (unsigned)((H->nseg + 7) / 8);
    // the second pass of Boolean list-output products (see k_pull_long)
    const bool two = Sr<T>::kPattern && SOUT && H->long_rest != nullptr;
    int4* rest = two ? H->long_rest : nullptr;
    unsigned int* rest_n = two ? H->long_rest_n : nullptr;
    if (vec)
        k_pull_long<T, MASK, SOUT, true><<<g, 256, 0, s>>>(H->nseg, H->nnz, H->seg, H->col, val, a, H->ws.ywork,
                                                           H->ws.yflag, H->long_part, H->long_hit, rest, rest_n);
    else
        k_pull_long<T, MASK, SOUT, false><<<g, 256, 0, s>>>(H->nseg, H->nnz, H->seg, H->col, val, a, H->ws.ywork,
                                                            H->ws.yflag, H->long_part, H->long_hit, rest, rest_n);
    if constexpr (Sr<T>::kPattern && SOUT) {
        if (two) {
            const unsigned gr = (unsigned)H->num_sms * 4;
            if (vec)
                k_pull_long_rest<T, MASK, true><<<gr, 256, 0, s>>>(rest, rest_n, H->nnz, H->col, a, H->ws.ywork,
                                                                   H->ws.yflag);
            else
                k_pull_long_rest<T, MASK, false><<<gr, 256, 0, s>>>(rest, rest_n, H->nnz, H->col, a, H->ws.ywork,
                                                                    H->ws.yflag);
        }
    }
    if (H->nmulti > 0 && !(Sr<T>::kPattern && SOUT)) {
        const unsigned gf = (unsigned)std::min<int64_t>((H->nmulti + 255) / 256, (int64_t)H->num_sms * 4);
        k_pull_long_fixup<T><<<gf, 256, 0, s>>>(H->nmulti, H->multi_row, H->multi_base, H->rowptr, H->long_part,
                                                H->long_hit, a, H->ws.ywork, H->ws.yflag, SOUT ? 1 : 0);
    }
}

template <class T, bool MASK, bool SOUT>
void launch_pull_warp_dtype(asv_matrix_s* H, const PullArg& a, bool vec, cudaStream_t s) {
    const int64_t m = H->m;
    const T* val = (const T*)H->val;
    void* ywork = H->ws.ywork;
    uint8_t* yt = H->ws.yflag;
        const int L = H->pull_lanes;
        if (m == 0) return;
        const int uu = H->pull_unroll >= 4 ? 4 : 2;
        const int rw = (32 / L) * ((L == 2) ? 2 : uu);
        const unsigned g = (unsigned)((m + 8 * rw - 1) / (8 * rw));
#define PW(LL)                                                                                                   \
    do {                                                                                                         \
        if (uu == 4) {                                                                                           \
            if (vec) k_pull_warp<T, MASK, SOUT, LL, true, 4><<<g, 256, 0, s>>>(m, H->nnz, H->rowptr, H->col, val, a, ywork, yt);  \
            else k_pull_warp<T, MASK, SOUT, LL, false, 4><<<g, 256, 0, s>>>(m, H->nnz, H->rowptr, H->col, val, a, ywork, yt); \
        } else {                                                                                                 \
            if (vec) k_pull_warp<T, MASK, SOUT, LL, true, 2><<<g, 256, 0, s>>>(m, H->nnz, H->rowptr, H->col, val, a, ywork, yt);  \
            else k_pull_warp<T, MASK, SOUT, LL, false, 2><<<g, 256, 0, s>>>(m, H->nnz, H->rowptr, H->col, val, a, ywork, yt); \
        }                                                                                                        \
    } while (0)
        switch (L) {
            case 2: PW(2); break;
            case 4: PW(4); break;
            case 8: PW(8); break;
            case 16: PW(16); break;
            default: PW(32); break;
        }
#undef PW
}

#define ASV_INSTANTIATE_PULL_WARP(T)                                                                   \
    template void launch_pull_warp_dtype<T, false, false>(asv_matrix_s*, const PullArg&, bool, cudaStream_t); \
    template void launch_pull_warp_dtype<T, false, true>(asv_matrix_s*, const PullArg&, bool, cudaStream_t);  \
    template void launch_pull_warp_dtype<T, true, false>(asv_matrix_s*, const PullArg&, bool, cudaStream_t);  \
    template void launch_pull_warp_dtype<T, true, true>(asv_matrix_s*, const PullArg&, bool, cudaStream_t);   \
    template void launch_pull_long_dtype<T, false, false>(asv_matrix_s*, const PullArg&, bool, cudaStream_t); \
    template void launch_pull_long_dtype<T, false, true>(asv_matrix_s*, const PullArg&, bool, cudaStream_t);  \
    template void launch_pull_long_dtype<T, true, false>(asv_matrix_s*, const PullArg&, bool, cudaStream_t);  \
    template void launch_pull_long_dtype<T, true, true>(asv_matrix_s*, const PullArg&, bool, cudaStream_t);

}  // namespace asv
