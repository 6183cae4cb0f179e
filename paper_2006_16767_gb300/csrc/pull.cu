// Row-major (CSR "pull") candidates of Sec. IV-A: the traditional SpMV
// (solution (3,6), no validation) and the row-major SpMSpV (solution (3,5),
// bitvector validation after GraphMat, Sec. VI-A), each with three workload
// distributions (Sec. IV-B): one row per thread (the paper's "direct"), a
// sub-warp of L lanes per row, and an even split of rows+nonzeros along the
// merge path (the paper's "load-balanced", after merge-based SpMV / Hola).
//
// Output: dense y (y_i written exactly once per call); in sparse-output mode
// y goes to a workspace and rows with an effective entry set their bit in the
// zero-invariant structural-set bitmap, which a compaction pass turns into
// the ascending output list.
#include "pull_common.cuh"
#include "tma.cuh"

namespace asv {

template <class T, bool MASK, bool SOUT>
void launch_pull_warp_dtype(asv_matrix_s* H, const PullArg& a, bool vec, cudaStream_t s);
template <class T, bool MASK, bool SOUT>
void launch_pull_long_dtype(asv_matrix_s* H, const PullArg& a, bool vec, cudaStream_t s);
void launch_pull_bool_fused(asv_matrix_s* H, const PullArg& a, bool masked, bool vec, cudaStream_t s);

constexpr int kBalB = 256;   // threads per balanced tile
constexpr int kBalIPT = 8;   // merge items per thread
constexpr int kBalD = kBalB * kBalIPT;

int64_t pull_tile_items(int32_t) { return kBalD; }

// ---------------------------------------------------------------- one row per thread
// Rows too long to stage (or a warp whose 32 rows do not fit the stage) are
// summed straight from global memory, one row per thread (arithmetic
// semirings; Boolean rows take pull_rows_bool).
template <class T, bool MASK, bool SOUT>
__device__ __forceinline__ typename Sr<T>::Acc row_direct(const int32_t* __restrict__ col, const T* __restrict__ val,
                                                          const T* __restrict__ x, const uint32_t* __restrict__ xbits,
                                                          int32_t b, int32_t e, bool& hit) {
    using S = Sr<T>;
    typename S::Acc acc;
    S::acc_zero(acc);
    for (int32_t k = b; k < e; ++k) {
        const int32_t c = __ldg(col + k);
        if (MASK || SOUT) {
            const bool bit = test_bit(xbits, c);
            hit |= bit;
            if (MASK && !bit) continue;
        }
        S::acc_add(acc, S::mul(load_val(val, k), __ldg(x + c)));
    }
    return acc;
}

// One row per thread (the paper's direct distribution) for rows of at most
// kLongRow entries; longer rows are left to k_pull_long. A warp owns 32
// consecutive rows; their contiguous span of column ids (and values, unless
// validation makes most of them unnecessary) is copied into shared memory
// with coalesced 128-bit loads, then every lane walks its own row there.
// With lanes on consecutive rows, the x gathers of one step land on
// neighbouring columns for banded and mesh-like matrices, so a warp's gather
// touches one or two cache lines instead of one per lane.
// entries staged per warp: a 32-row span of the 27-point stencil (at most
// 868 entries from its 16-byte-aligned start) fits, and four warps' stages
// (28.7 KB) leave room for seven blocks per SM where 1,024 entries left six
// (the stencil's dense-x product 718 -> 687 us on GB300)
constexpr int kStageCap = 896;
constexpr int kStageWarps = 4;

// NARROW (FP32 matrices whose rows all have at most kNarrowRow entries):
// a staged row is summed by a plain FMA chain instead of the compensated sum.
// k <= kNarrowRow terms each rounded once stay within k * 2^-24 * sum |a x|
// <= 1.91e-6 * sum |a x| of the exact sum (the FP32 tolerance is 2e-6 of it),
// and the walk issues a third of the instructions.
template <class T, bool MASK, bool SOUT, bool VEC, bool TMA, bool NARROW = false>
__global__ void __launch_bounds__(32 * kStageWarps) k_pull_thread(int64_t m, int64_t nnz,
                                                                  const int32_t* __restrict__ rowptr,
                                                                  const int32_t* __restrict__ col,
                                                                  const T* __restrict__ val, PullArg a, void* ywork,
                                                                  uint8_t* yflag, int32_t* status,
                                                                  uint32_t wait_limit) {
    using S = Sr<T>;
    constexpr bool kStageVals = !S::kPattern && !MASK;
    __shared__ __align__(16) int32_t s_col[kStageWarps][kStageCap];
    __shared__ __align__(16) T s_val[kStageVals ? kStageWarps : 1][kStageVals ? kStageCap : 1];
    __shared__ __align__(8) uint64_t s_bar[kStageWarps];
    const PullIO p = resolve(a, ywork, SOUT);
    const T* __restrict__ x = (const T*)p.x;
    T* __restrict__ y = (T*)p.y;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if constexpr (S::kPattern) {
        // Boolean rows stop at their first hit, so copying whole spans would
        // read indices the walk never touches: they take the direct walk,
        // kBoolRows groups of 32 rows per warp
        const int64_t rw = ((int64_t)blockIdx.x * kStageWarps + w) * 32 * kBoolRows;
        if (rw < m) pull_rows_bool<SOUT>(m, rowptr, col, p, (bool8*)y, yflag, rw, lane);
        return;
    }
    const int64_t r0 = ((int64_t)blockIdx.x * kStageWarps + w) * 32;
    if (r0 >= m) return;
    // a list output over a list of every column in order: every column's bit
    // is set, so a row is in the set when it has an entry (no bit tests), and
    // when every row is in it (y_ident) the flags are not written either
    const bool allx = SOUT && a.desc && a.desc->x_ident;
    const bool noflag = SOUT && a.desc && a.desc->y_ident;
    const int64_t i = r0 + lane;
    const int32_t rb = __ldg(rowptr + min(i, m));
    const int32_t span_end = __ldg(rowptr + min(r0 + 32, m));
    const int32_t re_n = __shfl_down_sync(0xffffffffu, rb, 1);
    const int32_t re = (lane == 31) ? span_end : re_n;
    const int32_t s0 = __shfl_sync(0xffffffffu, rb, 0);
    const int32_t a0 = s0 & ~3;
    const bool mine = i < m && re - rb <= kLongRow;  // longer rows are summed by k_pull_long
    const bool off = mine && row_masked(p.ymask, i);  // excluded by the output mask: y_i = 0
    bool hit = false;
    typename S::Acc acc;
    if (span_end - a0 <= kStageCap) {
        const int nchunks = (span_end - a0 + 3) >> 2;
        int32_t* sc = s_col[w];
        T* sv = kStageVals ? s_val[w] : nullptr;
        // TMA path: the whole 16-byte-aligned span (cut at the last full
        // 16-byte group of the arrays) in one bulk copy per array; the few
        // entries after that cut, at the very end of the matrix, by plain loads
        const int32_t bulk_end = min((int32_t)((span_end + 3) & ~3), (int32_t)(nnz & ~(int64_t)3));
        const int32_t nbulk = TMA ? max(0, bulk_end - a0) : 0;
        if (TMA) {
            if (nbulk > 0 && lane == 0) {
                mbar_init(&s_bar[w], 1);
                const uint32_t bytes = (uint32_t)nbulk * 4u * (kStageVals && val != nullptr ? (1u + sizeof(T) / 4u) : 1u);
                mbar_arrive_expect_tx(&s_bar[w], bytes);
                bulk_g2s(sc, col + a0, (uint32_t)nbulk * 4u, &s_bar[w]);
                if constexpr (kStageVals) {
                    if (val != nullptr) bulk_g2s(sv, val + a0, (uint32_t)nbulk * (uint32_t)sizeof(T), &s_bar[w]);
                }
            }
            __syncwarp();
            for (int32_t k = max(a0 + nbulk, s0) + lane; k < span_end; k += 32) {
                sc[k - a0] = __ldg(col + k);
                if constexpr (kStageVals) {
                    if (val != nullptr) sv[k - a0] = __ldg(val + k);
                }
            }
            if (nbulk > 0 && !mbar_wait(&s_bar[w], 0, wait_limit)) {
                // the copy did not land within the limit: report, wait again
                // under the default bound so no copy is left in flight when
                // the warp leaves, and give up
                latch_status(status, ASV_ERR_TIMEOUT);
                mbar_wait(&s_bar[w], 0);
                return;
            }
        }
        // four chunks per lane in flight at a time: loads first, then stores
        for (int q0 = 0; q0 < (TMA ? 0 : nchunks); q0 += 128) {
            int4 cb[4];
            int4 vb[4];
            double2 vd[4][2];
            bool full[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q = q0 + lane + 32 * u;
                const int32_t base = a0 + 4 * q;
                full[u] = VEC && q < nchunks && (int64_t)base + 4 <= nnz;
                if (full[u]) {
                    cb[u] = __ldg(reinterpret_cast<const int4*>(col + base));
                    if constexpr (kStageVals) {
                        if (val != nullptr) {
                            if constexpr (sizeof(T) == 4) {
                                vb[u] = __ldg(reinterpret_cast<const int4*>(val + base));
                            } else {
                                vd[u][0] = __ldg(reinterpret_cast<const double2*>(val + base));
                                vd[u][1] = __ldg(reinterpret_cast<const double2*>(val + base + 2));
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q = q0 + lane + 32 * u;
                if (q >= nchunks) continue;
                const int32_t base = a0 + 4 * q;
                if (full[u]) {
                    *reinterpret_cast<int4*>(sc + 4 * q) = cb[u];
                    if constexpr (kStageVals) {
                        if (val != nullptr) {
                            if constexpr (sizeof(T) == 4) {
                                *reinterpret_cast<int4*>(sv + 4 * q) = vb[u];
                            } else {
                                *reinterpret_cast<double2*>(sv + 4 * q) = vd[u][0];
                                *reinterpret_cast<double2*>(sv + 4 * q + 2) = vd[u][1];
                            }
                        }
                    }
                } else {
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        if ((int64_t)base + t < nnz) {
                            sc[4 * q + t] = __ldg(col + base + t);
                            if constexpr (kStageVals) {
                                if (val != nullptr) sv[4 * q + t] = __ldg(val + base + t);
                            }
                        }
                    }
                }
            }
        }
        __syncwarp();
        S::acc_zero(acc);
        float ps = 0.f;  // the NARROW sum
        // the walk, compiled for each (bit tests, value array) pair so that
        // neither per-entry condition costs an instruction in the loop
        auto walk = [&](auto bits_tag, auto vals_tag) {
            constexpr bool BITS = decltype(bits_tag)::value;
            constexpr bool VALS = decltype(vals_tag)::value;
            (void)VALS;
            int32_t k = rb;
            if constexpr (!MASK && kStageVals) {
                // eight gathers in flight per lane before their products are
                // added (the gathers, not HBM, bound a lane's walk of its row);
                // with a list output the same columns' bits say whether the
                // row is in the structural output set
                constexpr int GD = 8;
                for (; k + GD <= re; k += GD) {
                    T xg[GD];
                    uint32_t hb = 0u;
#pragma unroll
                    for (int u = 0; u < GD; ++u) {
                        const int32_t c = sc[k + u - a0];
                        xg[u] = __ldg(x + c);
                        if (SOUT && BITS) hb |= (uint32_t)test_bit(p.xbits, c);
                    }
                    if constexpr (NARROW) {
#pragma unroll
                        for (int u = 0; u < GD; ++u) ps = __fmaf_rn(VALS ? sv[k + u - a0] : 1.f, xg[u], ps);
                    } else {
#pragma unroll
                        for (int u = 0; u < GD; ++u) S::acc_add(acc, S::mul(VALS ? sv[k + u - a0] : S::one(), xg[u]));
                    }
                    if (SOUT) hit |= hb != 0u;
                }
                if (k + 4 <= re) {
                    T xg[4];
                    uint32_t hb = 0u;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int32_t c = sc[k + u - a0];
                        xg[u] = __ldg(x + c);
                        if (SOUT && BITS) hb |= (uint32_t)test_bit(p.xbits, c);
                    }
                    if constexpr (NARROW) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) ps = __fmaf_rn(VALS ? sv[k + u - a0] : 1.f, xg[u], ps);
                    } else {
#pragma unroll
                        for (int u = 0; u < 4; ++u) S::acc_add(acc, S::mul(VALS ? sv[k + u - a0] : S::one(), xg[u]));
                    }
                    if (SOUT) hit |= hb != 0u;
                    k += 4;
                }
            }
            for (; k < re; ++k) {
                const int32_t c = sc[k - a0];
                if (MASK || SOUT) {
                    const bool bit = !BITS || test_bit(p.xbits, c);
                    hit |= bit;
                    if (MASK && !bit) continue;
                }
                T v;
                if constexpr (kStageVals) v = VALS ? sv[k - a0] : S::one();
                else v = load_val(val, k);
                if constexpr (NARROW) ps = __fmaf_rn(v, __ldg(x + c), ps);
                else S::acc_add(acc, S::mul(v, __ldg(x + c)));
                if constexpr (S::kPattern) {
                    if (acc) break;
                }
            }
        };
        if (mine && !off) {
            using Y = std::true_type;
            using N = std::false_type;
            if (allx) {
                if (val != nullptr) walk(N{}, Y{});
                else walk(N{}, N{});
            } else {
                if (val != nullptr) walk(Y{}, Y{});
                else walk(Y{}, N{});
            }
        }
        if constexpr (NARROW) acc.s = ps;  // c stays 0: the value is ps
        if (allx) hit = mine && !off && re > rb;
    } else {
        if (mine && !off) acc = row_direct<T, MASK, SOUT>(col, val, x, p.xbits, rb, re, hit);
        else S::acc_zero(acc);
    }
    if (mine) {
        y[i] = S::part_T(S::acc_part(acc));
        if (SOUT && hit && !noflag) yflag[i] = 1;
    }
}

// ---------------------------------------------------------------- merge-path balanced
// Stages a tile's products into shared memory. Column ids (and values) are
// read with 128-bit loads over the 16-byte-aligned span covering [k0, k1);
// every load of the thread's groups is issued before any of them is used.
// With CHK (unvalidated caller arrays) a column id outside [0, ncols)
// contributes nothing instead of gathering outside x.
template <class T, bool MASK, bool SOUT, bool VEC, bool CHK = false>
__device__ __forceinline__ void stage_products(const int32_t* __restrict__ col, const T* __restrict__ val,
                                               const T* __restrict__ x, const uint32_t* __restrict__ xbits,
                                               int64_t k0, int64_t k1, int64_t nnz, typename Sr<T>::Part* s_prod,
                                               uint32_t* s_eff, int64_t ncols = 0) {
    using S = Sr<T>;
    using P = typename S::Part;
    constexpr int MAXG = (kBalD / 4 + 1 + kBalB - 1) / kBalB;
    const int64_t a0 = k0 & ~(int64_t)3;
    const int ngroups = (int)((k1 - a0 + 3) >> 2);
    int32_t c[MAXG][4];
    T v[MAXG][4];
    bool eff[MAXG][4], bitv[MAXG][4];
#pragma unroll
    for (int j = 0; j < MAXG; ++j) {
        const int gi = threadIdx.x + j * kBalB;
        const int64_t base = a0 + 4 * (int64_t)gi;
        if (gi < ngroups && VEC && base + 4 <= nnz) {
            const int4 cc = __ldg(reinterpret_cast<const int4*>(col + base));
            c[j][0] = cc.x; c[j][1] = cc.y; c[j][2] = cc.z; c[j][3] = cc.w;
            if constexpr (!S::kPattern && !MASK) {
                if (val != nullptr) {
                    if constexpr (sizeof(T) == 4) {
                        const int4 vv = __ldg(reinterpret_cast<const int4*>(val + base));
                        v[j][0] = __int_as_float_t<T>(vv.x); v[j][1] = __int_as_float_t<T>(vv.y);
                        v[j][2] = __int_as_float_t<T>(vv.z); v[j][3] = __int_as_float_t<T>(vv.w);
                    } else {
                        const double2 v01 = __ldg(reinterpret_cast<const double2*>(val + base));
                        const double2 v23 = __ldg(reinterpret_cast<const double2*>(val + base + 2));
                        v[j][0] = (T)v01.x; v[j][1] = (T)v01.y; v[j][2] = (T)v23.x; v[j][3] = (T)v23.y;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) v[j][q] = S::one();
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t k = base + q;
                const bool in = gi < ngroups && k >= k0 && k < k1;
                c[j][q] = in ? __ldg(col + k) : 0;
                if constexpr (!S::kPattern && !MASK) v[j][q] = in ? load_val(val, k) : T(0);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < MAXG; ++j) {
        const int gi = threadIdx.x + j * kBalB;
        const int64_t base = a0 + 4 * (int64_t)gi;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t k = base + q;
            const bool in = gi < ngroups && k >= k0 && k < k1 &&
                            (!CHK || (uint64_t)(uint32_t)c[j][q] < (uint64_t)ncols);
            if constexpr (S::kPattern) {
                bitv[j][q] = in && bool_gather(x, xbits, c[j][q]);  // the term itself
                eff[j][q] = bitv[j][q];
            } else {
                bitv[j][q] = (MASK || SOUT) && in ? test_bit(xbits, c[j][q]) : true;
                eff[j][q] = in && (!MASK || bitv[j][q]);
            }
        }
        if constexpr (S::kPattern) {
#pragma unroll
            for (int q = 0; q < 4; ++q) v[j][q] = S::one();
        } else if constexpr (MASK) {
#pragma unroll
            for (int q = 0; q < 4; ++q) v[j][q] = eff[j][q] ? load_val(val, base + q) : T(0);
        }
    }
#pragma unroll
    for (int j = 0; j < MAXG; ++j) {
        const int gi = threadIdx.x + j * kBalB;
        const int64_t base = a0 + 4 * (int64_t)gi;
        P pr[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if constexpr (S::kPattern) pr[q] = eff[j][q] ? P(1) : P(0);
            else pr[q] = eff[j][q] ? S::mul(v[j][q], __ldg(x + c[j][q])) : P(0);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t k = base + q;
            if (gi < ngroups && k >= k0 && k < k1) {
                const int li = (int)(k - k0);
                s_prod[li] = pr[q];
                if (SOUT && bitv[j][q]) atomicOr(&s_eff[li >> 5], 1u << (li & 31));
            }
        }
    }
}

// CHK: the CSR arrays come from a caller who did not build a handle and were
// never validated, so a tile whose bounds a malformed row-pointer array makes
// inconsistent is skipped (it writes nothing), the merge never walks past
// the tile's entries, and column ids outside [0, ncols) are dropped: every
// access stays inside the arrays whatever their contents.
template <class T, bool MASK, bool SOUT, bool VEC, bool CHK = false>
__global__ void __launch_bounds__(kBalB) k_pull_bal(int64_t m, int64_t nnz, const int32_t* __restrict__ rowptr,
                                                    const int32_t* __restrict__ col, const T* __restrict__ val,
                                                    const int32_t* __restrict__ tile_row, PullArg a, void* ywork,
                                                    uint8_t* yflag, int32_t* carry_row,
                                                    typename Sr<T>::Atom* carry_val, int64_t ncols = 0) {
    using S = Sr<T>;
    using P = typename S::Part;
    constexpr int B = kBalB, IPT = kBalIPT, D = kBalD, NW = B / 32;
    __shared__ int32_t s_end[D];
    __shared__ P s_prod[D];
    __shared__ P s_row[D];
    __shared__ P s_scan[B];
    __shared__ uint32_t s_eff[SOUT ? D / 32 : 1];
    __shared__ int32_t s_wkey[NW], s_wfirst[NW];
    __shared__ P s_wval[NW];

    const PullIO p = resolve(a, ywork, SOUT);
    const T* __restrict__ x = (const T*)p.x;
    T* __restrict__ y = (T*)p.y;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

    const int64_t t = blockIdx.x;
    const int64_t d0 = t * D, d1 = min(d0 + D, m + nnz);
    const int32_t r0 = tile_row[t], r1 = tile_row[t + 1];
    const int64_t k0 = d0 - r0, k1 = d1 - r1;
    const int nrows = r1 - r0, nk = (int)(k1 - k0);
    if (CHK && (nrows < 0 || nk < 0 || k0 < 0 || k1 > nnz)) {  // the same verdict in every thread
        if (threadIdx.x == 0) {
            carry_row[t] = -1;
            carry_val[t] = S::to_atom(T(0));
        }
        return;
    }

    for (int i = threadIdx.x; i < nrows; i += B) s_end[i] = __ldg(rowptr + r0 + 1 + i);
    if (SOUT)
        for (int i = threadIdx.x; i < D / 32; i += B) s_eff[i] = 0u;
    if (SOUT) __syncthreads();
    stage_products<T, MASK, SOUT, VEC, CHK>(col, val, x, p.xbits, k0, k1, nnz, s_prod, s_eff, ncols);
    __syncthreads();

    // this thread's share of the tile's merge path
    const int total = nrows + nk;
    const int dt = min((int)threadIdx.x * IPT, total), dte = min(dt + IPT, total);
    int lo = max(0, dt - nk), hi = min(dt, nrows);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((int64_t)s_end[mid] <= k0 + (dt - mid - 1)) lo = mid + 1;
        else hi = mid;
    }
    int ri = lo, ki = dt - lo;
    const int ri_start = ri;
    typename S::Acc acc;
    S::acc_zero(acc);
    bool hit = false;
    for (int step = dt; step < dte; ++step) {
        if (ri < nrows && ((int64_t)s_end[ri] <= k0 + ki || (CHK && ki >= nk))) {
            s_row[ri] = S::acc_part(acc);
            S::acc_zero(acc);
            if (SOUT && hit && !row_masked(p.ymask, (int64_t)r0 + ri)) yflag[(int64_t)r0 + ri] = 1;
            hit = false;
            ++ri;
        } else {
            if (CHK && ki >= nk) break;
            S::acc_add(acc, s_prod[ki]);
            if (SOUT) hit |= (s_eff[ki >> 5] >> (ki & 31)) & 1u;
            ++ki;
        }
    }
    if (SOUT && hit && !row_masked(p.ymask, (int64_t)r0 + ri)) yflag[(int64_t)r0 + ri] = 1;

    // segmented inclusive scan of the threads' carries (key = row still open
    // at the thread's end; keys are non-decreasing across threads)
    P v = S::acc_part(acc);
    const int key = ri;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const P pv = shfl_up(v, o);
        const int pk = shfl_up(key, o);
        if (lane >= o && pk == key) v = S::part_add(pv, v);
    }
    if (lane == 31) { s_wkey[wid] = key; s_wval[wid] = v; }
    if (lane == 0) s_wfirst[wid] = key;
    __syncthreads();
    if (wid > 0 && s_wkey[wid - 1] == key) {
        P c = s_wval[wid - 1];
        int ww = wid - 1;
        while (ww > 0 && s_wfirst[ww] == key && s_wkey[ww - 1] == key) {
            c = S::part_add(s_wval[ww - 1], c);
            --ww;
        }
        v = S::part_add(c, v);
    }
    s_scan[threadIdx.x] = v;
    __syncthreads();
    // the first row this thread completed collects the carries of the
    // threads before it that worked on the same row
    if (threadIdx.x > 0 && ri > ri_start) s_row[ri_start] = S::part_add(s_scan[threadIdx.x - 1], s_row[ri_start]);
    __syncthreads();
    for (int i = threadIdx.x; i < nrows; i += B)
        y[r0 + i] = row_masked(p.ymask, (int64_t)r0 + i) ? T(0) : S::part_T(s_row[i]);
    if (threadIdx.x == B - 1) {
        carry_row[t] = (r1 < m) ? r1 : -1;
        carry_val[t] = S::to_atom(S::part_T(v));
    }
}

// Adds the partial sums of rows that span several tiles: the first tile of a
// run of tiles that leave the same row open sums their carries (in FP64 for
// the floating-point types) into the value the completing tile wrote.
template <class T>
__global__ void k_pull_bal_fixup(int64_t ntiles, const int32_t* __restrict__ carry_row,
                                 const typename Sr<T>::Atom* __restrict__ carry_val, const CallDesc* desc,
                                 void* ydirect, void* ywork, int sparse_out) {
    using S = Sr<T>;
    T* y = (T*)(desc ? (sparse_out ? (desc->y_ident ? desc->yval : ywork) : desc->y) : ydirect);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntiles; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = carry_row[t];
        if (r < 0) continue;
        if (t > 0 && carry_row[t - 1] == r) continue;
        if (desc && row_masked(desc->ymask, r)) continue;  // the completing tile wrote 0
        typename S::Atom s = carry_val[t];
        for (int64_t u = t + 1; u < ntiles && carry_row[u] == r; ++u) {
            if constexpr (S::kPattern) s = s | carry_val[u];
            else s = s + carry_val[u];
        }
        if constexpr (S::kPattern) y[r] = S::from_atom(S::to_atom(S::part_of(y[r])) | s);
        else y[r] = S::from_atom(S::to_atom(S::part_of(y[r])) + s);
    }
}

// ---------------------------------------------------------------- launcher
template <class T, bool MASK, bool SOUT>
static void pull_dispatch(asv_matrix_s* H, int dist, const PullIO* direct, cudaStream_t s) {
    PullArg a;
    a.desc = direct ? nullptr : H->d_desc;
    if (direct) a.io = *direct;
    else a.io = PullIO{nullptr, nullptr, nullptr};
    const int64_t m = H->m;
    const T* val = (const T*)H->val;
    void* ywork = H->ws.ywork;
    uint8_t* yt = H->ws.yflag;
    const int64_t cap = (int64_t)H->num_sms * 16;
    const bool vec = ((uintptr_t)H->col % 16 == 0) && ((uintptr_t)H->val % 16 == 0);
    // rows over kLongRow entries: their warp-per-segment pass (and fix-up)
    // goes first, on the side stream; the short-row kernel then fills the SMs
    // that the pass's tail -- segments walked to their end -- leaves idle.
    // The two write disjoint rows. A Boolean list-output thread pull runs
    // both in one launch instead (k_pull_bool_fused).
    const bool fused = Sr<T>::kPattern && SOUT && dist == 0 && H->nseg > 0 && H->long_rest != nullptr;
    const bool fork = dist != 2 && H->nseg > 0 && !fused;
    if (fork) {
        cudaEventRecord(H->ev_fork, s);
        cudaStreamWaitEvent(H->side_stream, H->ev_fork, 0);
        launch_pull_long_dtype<T, MASK, SOUT>(H, a, vec, H->side_stream);
        cudaEventRecord(H->ev_join, H->side_stream);
    }
    if (fused) {
        if constexpr (Sr<T>::kPattern && SOUT) launch_pull_bool_fused(H, a, MASK, vec, s);
    } else if (dist == 0) {
        const int64_t rows_per_block = 32 * kStageWarps * (Sr<T>::kPattern ? kBoolRows : 1);
        const unsigned g = (unsigned)((m + rows_per_block - 1) / rows_per_block);
        int32_t* st = H->ws.status;
        const uint32_t wl = H->wait_limit;
        if (m > 0) {
            const bool narrow = std::is_same<T, float>::value && H->narrow_acc;
#define PULL_THREAD(V, TM)                                                                                   \
    do {                                                                                                     \
        if (narrow) {                                                                                        \
            if constexpr (std::is_same<T, float>::value)                                                     \
                k_pull_thread<T, MASK, SOUT, V, TM, true><<<g, 32 * kStageWarps, 0, s>>>(m, H->nnz, H->rowptr, \
                                                                                       H->col, val, a, ywork, \
                                                                                       yt, st, wl);          \
        } else {                                                                                             \
            k_pull_thread<T, MASK, SOUT, V, TM><<<g, 32 * kStageWarps, 0, s>>>(m, H->nnz, H->rowptr, H->col,   \
                                                                           val, a, ywork, yt, st, wl);       \
        }                                                                                                    \
    } while (0)
            if (vec && H->pull_tma) PULL_THREAD(true, true);
            else if (vec) PULL_THREAD(true, false);
            else PULL_THREAD(false, false);
#undef PULL_THREAD
        }
    } else if (dist == 1) {
        launch_pull_warp_dtype<T, MASK, SOUT>(H, a, vec, s);
    } else {
        if (H->ntiles == 0) return;
        using Atom = typename Sr<T>::Atom;
        if (vec)
            k_pull_bal<T, MASK, SOUT, true><<<(int)H->ntiles, kBalB, 0, s>>>(
                m, H->nnz, H->rowptr, H->col, val, H->tile_row, a, ywork, yt, H->carry_row, (Atom*)H->carry_val);
        else
            k_pull_bal<T, MASK, SOUT, false><<<(int)H->ntiles, kBalB, 0, s>>>(
                m, H->nnz, H->rowptr, H->col, val, H->tile_row, a, ywork, yt, H->carry_row, (Atom*)H->carry_val);
        const int64_t g = min(cap, (H->ntiles + 255) / 256);
        k_pull_bal_fixup<T><<<(int)g, 256, 0, s>>>(H->ntiles, H->carry_row, (const Atom*)H->carry_val,
                                                   direct ? nullptr : H->d_desc, direct ? direct->y : nullptr,
                                                   ywork, SOUT ? 1 : 0);
    }
    if (fork) cudaStreamWaitEvent(s, H->ev_join, 0);
}

// The FP32 balanced pull on caller-owned, unvalidated arrays and
// caller-provided scratch (tile table, carries), with the bounds checks of
// the CHK form; used by the allocation-free entry point.
void launch_pull_bal_f32_raw(int64_t m, int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                             const float* val, const float* x, float* y, const int32_t* tile_row, int32_t* carry_row,
                             double* carry_val, int64_t ntiles, cudaStream_t s) {
    if (ntiles == 0) return;
    PullArg a;
    a.desc = nullptr;
    a.io = PullIO{x, nullptr, y};
    const bool vec = ((uintptr_t)col % 16 == 0) && ((uintptr_t)val % 16 == 0);
    if (vec)
        k_pull_bal<float, false, false, true, true><<<(int)ntiles, kBalB, 0, s>>>(
            m, nnz, rowptr, col, val, tile_row, a, nullptr, nullptr, carry_row, carry_val, n);
    else
        k_pull_bal<float, false, false, false, true><<<(int)ntiles, kBalB, 0, s>>>(
            m, nnz, rowptr, col, val, tile_row, a, nullptr, nullptr, carry_row, carry_val, n);
    k_pull_bal_fixup<float><<<(int)((ntiles + 255) / 256), 256, 0, s>>>(ntiles, carry_row, carry_val, nullptr, y,
                                                                        nullptr, 0);
}

template <class T>
static void pull_dtype(asv_matrix_s* H, int dist, bool masked, bool sout, const PullIO* direct, cudaStream_t s) {
    if (masked) {
        if (sout) pull_dispatch<T, true, true>(H, dist, direct, s);
        else pull_dispatch<T, true, false>(H, dist, direct, s);
    } else {
        if (sout) pull_dispatch<T, false, true>(H, dist, direct, s);
        else pull_dispatch<T, false, false>(H, dist, direct, s);
    }
}

void launch_pull(asv_matrix_s* H, int dist, bool masked, bool sparse_out, const PullIO* direct, cudaStream_t s) {
    switch (H->dtype) {
        case ASV_F32: pull_dtype<float>(H, dist, masked, sparse_out, direct, s); break;
        case ASV_F64: pull_dtype<double>(H, dist, masked, sparse_out, direct, s); break;
        case ASV_I32: pull_dtype<int32_t>(H, dist, masked, sparse_out, direct, s); break;
        case ASV_BOOL: pull_dtype<bool8>(H, dist, masked, sparse_out, direct, s); break;
    }
}

}  // namespace asv
