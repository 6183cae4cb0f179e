// Per-call vector work of the runtime procedure (Sec. VI-C): the feature pass
// over x (nnz_x, x_sparsity, nnz_s, m_sparsity of Table 1) that also builds
// x's bitmap (the bitvector of Sec. VI-A) and fills the call descriptor;
// sparse<->dense conversion of x (done only inside the branches that need it);
// ordered stream compaction; and write-out of the push kernels' accumulators.
#include "internal.h"
#include "prims.cuh"

namespace asv {

// Block totals of the feature pass go to zero-invariant counters; the last
// block to finish (ticket) publishes them to the descriptor and re-zeroes.
__device__ __forceinline__ void publish_desc(CallDesc* desc, const DescInit& di, unsigned long long nx,
                                             unsigned long long ns, unsigned long long nh, int64_t n, int64_t nnz) {
    desc->x_dense = di.x_dense;
    desc->xbits = di.xbits;
    desc->xidx = di.xidx;
    desc->xval = di.xval;
    desc->nnz_x = (int64_t)nx;
    desc->nnz_s = (int64_t)ns;
    desc->y = di.y;
    desc->yidx = di.yidx;
    desc->yval = di.yval;
    desc->nnz_y = di.nnz_y;
    desc->y_cap = di.y_cap;
    desc->user_x_dense = di.user_x_dense;
    desc->user_xidx = di.user_xidx;
    desc->user_xval = di.user_xval;
    desc->out_mode = di.out_mode;
    desc->x_sparse = di.x_sparse;
    desc->ymask = di.ymask;
    desc->nhub = (int64_t)nh;
    desc->x_ident = 0;
    desc->y_ident = 0;
    desc->vfeat[0] = (double)nx;
    desc->vfeat[1] = n > 0 ? (double)nx / (double)n : 0.0;
    desc->vfeat[2] = (double)ns;
    desc->vfeat[3] = nnz > 0 ? (double)ns / (double)nnz : 0.0;
}

// The hub-column queue's length as the previous call left it, read by
// thread 0 of every block at the start of the feature pass (only the push
// kernels, which run after the pass, change it), so the block that resets
// the queue does not wait for the read.
__device__ __forceinline__ unsigned hub_queue_len(const SelectArg& sa) {
    return (threadIdx.x == 0 && sa.lcol_n) ? *(volatile unsigned int*)sa.lcol_n : 0u;
}

// Returns the push kernels' hub-column queue and the Boolean pull's
// long-row piece queue of the previous call to their empty state (one
// block, all its threads; nq from hub_queue_len, valid in thread 0).
template <int B>
__device__ __forceinline__ void reset_hub_queue(const SelectArg& sa, unsigned nq) {
    if (threadIdx.x == 0 && sa.long_rest_n) *sa.long_rest_n = 0u;
    if (!sa.lcol_n) return;
    __shared__ int32_t s_nq;
    if (threadIdx.x == 0) s_nq = min((int32_t)nq, sa.lcol_cap);
    __syncthreads();
    for (int32_t i = threadIdx.x; i < s_nq; i += B) sa.lcol[i] = make_int2(-1, 0);
    if (threadIdx.x == 0) *sa.lcol_n = 0u;
}

// `blocks` is the number of blocks that take part (all of them call this);
// the one that draws the last ticket publishes (a pass of one block, a short
// list, publishes its own totals and leaves the counters and the ticket
// alone). ch counts the listed columns longer than kLongSeg.
// With ident, cm counts the list entries t whose column is not t: none means
// the list is every column in order, and the call's pull kernels read its
// values in place.
template <int B>
__device__ __forceinline__ void finish_counts(unsigned long long cx, unsigned long long cs, unsigned long long ch,
                                              unsigned long long* counters, unsigned int* ticket, CallDesc* desc,
                                              const DescInit& di, int64_t n, int64_t nnz, int32_t* status,
                                              const SelectArg& sa, unsigned blocks, TreeNode* sn, unsigned nq,
                                              bool ident = false, unsigned long long cm = 0) {
    __shared__ unsigned long long sm[B / 32 + 1];
    __shared__ bool last;
    __shared__ double s_vf[4];  // the published vector features, for the selector
    cx = block_reduce_sum<B>(cx, sm);
    cs = block_reduce_sum<B>(cs, sm);
    ch = block_reduce_sum<B>(ch, sm);
    if (ident) cm = block_reduce_sum<B>(cm, sm);
    const bool alone = blocks == 1;
    if (threadIdx.x == 0) {
        if (alone) {
            last = true;
        } else {
            if (cx) atomicAdd(&counters[0], cx);
            if (cs) atomicAdd(&counters[1], cs);
            if (ch) atomicAdd(&counters[2], ch);
            if (cm) atomicAdd(&counters[3], cm);
            __threadfence();
            last = atomicAdd(ticket, 1u) == blocks - 1;
        }
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        unsigned long long nx = cx, ns = cs, nh = ch, nm = cm;
        if (!alone) {
            __threadfence();
            nx = atomicExch(&counters[0], 0ull);
            ns = atomicExch(&counters[1], 0ull);
            nh = atomicExch(&counters[2], 0ull);
            nm = atomicExch(&counters[3], 0ull);
        }
        // a list with repeated or out-of-range entries could exceed the
        // workspaces sized for nnz_x <= n and nnz_s <= nnz: clamp and report
        if (nx > (unsigned long long)n || ns > (unsigned long long)nnz) {
            latch_status(status, ASV_ERR_ARG);
            nx = nx > (unsigned long long)n ? (unsigned long long)n : nx;
            ns = ns > (unsigned long long)nnz ? (unsigned long long)nnz : ns;
        }
        publish_desc(desc, di, nx, ns, nh < nx ? nh : nx, n, nnz);
        if (ident && nm == 0 && nx == (unsigned long long)n) {
            desc->x_ident = 1;
            desc->x_dense = di.xval;
        }
        // x reaches every column and no row is empty: every row is in the
        // structural output set
        if (di.y_ident_ok && di.ymask == nullptr && nx == (unsigned long long)n) desc->y_ident = 1;
        s_vf[0] = (double)nx;
        s_vf[1] = n > 0 ? (double)nx / (double)n : 0.0;
        s_vf[2] = (double)ns;
        s_vf[3] = nnz > 0 ? (double)ns / (double)nnz : 0.0;
        if (!alone) {
            __threadfence();
            atomicExch(ticket, 0u);
        }
    }
    // the last block returns the push kernels' hub-column queue of the
    // previous call to its empty state
    if (last) reset_hub_queue<B>(sa, nq);
    // the last block also walks the selector's trees (Sec. VI-B), staged at
    // the start of the pass, so the choice is ready when the feature pass ends
    if (last && sa.enabled) {
        __syncthreads();
        run_selector(sa, desc, sn, s_vf);
    }
}

// Four consecutive elements of x as raw words, with one 128-bit (for bytes,
// 32-bit; for 8-byte values, two 128-bit) load, issued ahead of their use.
template <class T>
struct Raw4 {
    typename std::conditional<sizeof(T) == 8, double4, typename std::conditional<sizeof(T) == 4, int4, uchar4>::type>::type v;
};

template <class T>
__device__ __forceinline__ Raw4<T> load4_raw(const T* __restrict__ x, int64_t j) {
    Raw4<T> r;
    if constexpr (sizeof(T) == 8) {
        const double2 a = __ldg(reinterpret_cast<const double2*>(x + j));
        const double2 b = __ldg(reinterpret_cast<const double2*>(x + j + 2));
        r.v = make_double4(a.x, a.y, b.x, b.y);
    } else if constexpr (sizeof(T) == 4) {
        r.v = __ldg(reinterpret_cast<const int4*>(x + j));
    } else {
        r.v = __ldg(reinterpret_cast<const uchar4*>(x + j));
    }
    return r;
}

// Bit q of the result: element q of the four is nonzero.
template <class T>
__device__ __forceinline__ unsigned raw_nib(const Raw4<T>& r) {
    if constexpr (sizeof(T) == 8) {
        return (unsigned)(r.v.x != 0.0) | ((unsigned)(r.v.y != 0.0) << 1) | ((unsigned)(r.v.z != 0.0) << 2) |
               ((unsigned)(r.v.w != 0.0) << 3);
    } else if constexpr (sizeof(T) == 4) {
        return (unsigned)Sr<T>::nz(*reinterpret_cast<const T*>(&r.v.x)) |
               ((unsigned)Sr<T>::nz(*reinterpret_cast<const T*>(&r.v.y)) << 1) |
               ((unsigned)Sr<T>::nz(*reinterpret_cast<const T*>(&r.v.z)) << 2) |
               ((unsigned)Sr<T>::nz(*reinterpret_cast<const T*>(&r.v.w)) << 3);
    } else {
        return (unsigned)(r.v.x != 0) | ((unsigned)(r.v.y != 0) << 1) | ((unsigned)(r.v.z != 0) << 2) |
               ((unsigned)(r.v.w != 0) << 3);
    }
}

// Dense x: a warp covers 128 elements (four bitmap words) per step, lane l
// the four elements 4l..4l+3; the nibbles of eight lanes form one word. The
// degree of every nonzero column comes from colptr; block totals go to the
// ticketed counters.
template <class T, int B>
__global__ void __launch_bounds__(B, 6) k_feat_dense(const T* __restrict__ x, int64_t n, const int32_t* __restrict__ colptr,
                                                  uint32_t* xbits, unsigned long long* counters, unsigned int* ticket,
                                                  CallDesc* desc, DescInit di, int64_t nnz, int32_t* status,
                                                  SelectArg sa) {
    __shared__ TreeNode sn[kTreeWindow];
    // the selector's trees are staged while the pass runs (the last block
    // walks them)
    if (sa.enabled) stage_window<B>(sa, sn);
    const unsigned nq = hub_queue_len(sa);
    const bool VEC = ((uintptr_t)x & 15) == 0;
    const int lane = threadIdx.x & 31;
    const int64_t nwords = (n + 31) >> 5;
    const int64_t nsuper = (n + 127) >> 7;
    const int64_t gw = (int64_t)blockIdx.x * (B / 32) + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * (B / 32);
    unsigned long long cx = 0, cs = 0, ch = 0;
    // each lane's next 16 bytes of x are loaded before the current ones are
    // used, so a warp keeps two loads in flight through its ~18 steps (three,
    // with five blocks per SM instead of six, measured no faster: the
    // stencil's dense-x calls 0.3-4 % slower)
    Raw4<T> cur{};
    bool cur_vec = gw < nsuper && VEC && gw * 128 + lane * 4 + 4 <= n;
    if (cur_vec) cur = load4_raw(x, gw * 128 + lane * 4);
    for (int64_t sw = gw; sw < nsuper; sw += nw) {
        const int64_t j0 = sw * 128 + lane * 4;
        const int64_t swn = sw + nw, jn = swn * 128 + lane * 4;
        const bool nxt_vec = swn < nsuper && VEC && jn + 4 <= n;
        Raw4<T> nxt{};
        if (nxt_vec) nxt = load4_raw(x, jn);
        unsigned nib = 0u;
        bool nz[4];
        if (cur_vec) {
            nib = raw_nib(cur);
#pragma unroll
            for (int q = 0; q < 4; ++q) nz[q] = (nib >> q) & 1u;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) nz[q] = (j0 + q < n) && Sr<T>::nz(__ldg(x + j0 + q));
            nib = (unsigned)nz[0] | ((unsigned)nz[1] << 1) | ((unsigned)nz[2] << 2) | ((unsigned)nz[3] << 3);
        }
        cur = nxt;
        cur_vec = nxt_vec;
        // a fully nonzero stretch of 128 columns: two boundary reads give its
        // degree sum, so a dense x does not stream all of colptr
        if (__all_sync(0xffffffffu, nib == 0xFu && j0 + 4 <= n)) {
            int32_t span = 0;
            if (lane == 0) span = __ldg(colptr + sw * 128 + 128) - __ldg(colptr + sw * 128);
            if (lane == 0) cs += (unsigned long long)span;
            // a stretch longer than one hub may hold hubs: count them
            if (__shfl_sync(0xffffffffu, span, 0) > kLongSeg) {
                const int4 cp = __ldg(reinterpret_cast<const int4*>(colptr + j0));
                const int32_t c4 = __ldg(colptr + j0 + 4);
                ch += (cp.y - cp.x > kLongSeg) + (cp.z - cp.y > kLongSeg) + (cp.w - cp.z > kLongSeg) +
                      (c4 - cp.w > kLongSeg);
            }
        } else if (nib) {
            if (j0 + 4 <= n) {
                const int4 cp = __ldg(reinterpret_cast<const int4*>(colptr + j0));
                const int32_t c4 = __ldg(colptr + j0 + 4);
                const int32_t d[4] = {cp.y - cp.x, cp.z - cp.y, cp.w - cp.z, c4 - cp.w};
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (nz[q]) {
                        cs += (unsigned long long)d[q];
                        ch += d[q] > kLongSeg;
                    }
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (nz[q]) {
                        const int32_t d = __ldg(colptr + j0 + q + 1) - __ldg(colptr + j0 + q);
                        cs += (unsigned long long)d;
                        ch += d > kLongSeg;
                    }
            }
        }
        unsigned wv = nib << (4 * (lane & 7));
        wv |= __shfl_xor_sync(0xffffffffu, wv, 1);
        wv |= __shfl_xor_sync(0xffffffffu, wv, 2);
        wv |= __shfl_xor_sync(0xffffffffu, wv, 4);
        if ((lane & 7) == 0) {
            const int64_t w = sw * 4 + (lane >> 3);
            if (w < nwords) {
                xbits[w] = wv;
                cx += __popc(wv);
            }
        }
    }
    finish_counts<B>(cx, cs, ch, counters, ticket, desc, di, n, nnz, status, sa, gridDim.x, sn, nq);
}

// Sparse x: nnz_s = sum of the listed columns' lengths.
template <int B>
__global__ void __launch_bounds__(B) k_feat_sparse(const int64_t* __restrict__ nnz_x_dev, const int32_t* __restrict__ xidx,
                                                   const int32_t* __restrict__ colptr, unsigned long long* counters,
                                                   unsigned int* ticket, CallDesc* desc, DescInit di, int64_t n,
                                                   int64_t nnz, int32_t* status, SelectArg sa, int64_t hub_cols) {
    __shared__ TreeNode sn[kTreeWindow];
    int64_t nx = *nnz_x_dev;
    const unsigned nq = hub_queue_len(sa);
    if (nx < 0) nx = 0;
    if (nx > n) nx = n + 1;  // reported and clamped when the totals are published
    // a list of n distinct columns is every column: its effective entries are
    // all nnz entries and its hubs the matrix's long columns, so one block
    // publishes them without a gather
    const bool every = nx == n;
    // such a list with values is also checked for being every column in
    // order (xidx[t] = t, which an ascending list of every column is): the
    // pull kernels then read its values in place, with no scatter into the
    // dense workspace (a pass over the indices instead of a pass over indices
    // and values plus a write and a clear of the workspace)
    const bool ident = every && di.xval != nullptr && n > 0;
    // only the blocks the list reaches take part (a short list costs one block)
    const unsigned blocks =
        every && !ident ? 1u : (unsigned)max((int64_t)1, min((int64_t)gridDim.x, (min(nx, n) + B - 1) / B));
    // block 0 always takes part: its copy of the selector's trees is issued
    // together with the load of nnz_x
    if (sa.enabled && blockIdx.x == 0) stage_window<B>(sa, sn);
    if (blockIdx.x >= blocks) return;
    if (sa.enabled && blockIdx.x != 0) stage_window<B>(sa, sn);
    // Lazy, cost-ordered evaluation (Sec. VI-C: cheap features first): a list
    // gives nnz_x and x_sparsity for free, while nnz_s and m_sparsity cost a
    // pass of gathers over its columns' pointers. When the call format's trees
    // start with a free feature, every taking part block walks them with the
    // free features alone; if the path needs no other feature and the chosen
    // kernel reads neither nnz_s nor the hub count (the pull kernels and the
    // warp push with atomics), block 0 publishes the call without them and
    // the pass ends there.
    if (sa.enabled && sa.lazy && nx <= n && !ident) {
        __shared__ double s_f[13];
        __shared__ int s_kid;
        if (threadIdx.x == 0) {
#pragma unroll
            for (int q = 0; q < 9; ++q) s_f[q] = sa.mf[q];
            s_f[9] = (double)nx;
            s_f[10] = n > 0 ? (double)nx / (double)n : 0.0;
            s_f[11] = s_f[12] = 0.0;
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            int kid = pick_kernel(sa, sn, s_f, 11);
            if (!(kid >= ASV_K_PULL_THREAD && kid <= ASV_K_MPULL_BAL) && kid != ASV_K_PUSH_WARP_ATOM) kid = -1;
            if (threadIdx.x == 0) s_kid = kid;
        }
        __syncthreads();
        const int kid = s_kid;
        if (kid >= 0) {
            if (blockIdx.x == 0) {
                if (threadIdx.x == 0) {
                    publish_desc(desc, di, (unsigned long long)nx, 0ull, 0ull, n, nnz);
                    desc->nnz_s = -1;  // not computed
                    desc->vfeat[2] = desc->vfeat[3] = -1.0;
                    commit_kernel(sa, desc, kid);
                }
                reset_hub_queue<B>(sa, nq);
            }
            return;
        }
    }
    // four list entries per thread in flight: their column lengths are
    // independent gathers (eight consecutive entries per thread, read with
    // two 16-byte loads, measured faster on a 16.8M-entry list, 861 -> 853 us
    // for its whole call, but slower on the lists of 10^3 - 10^6 entries that
    // BFS levels and sparse products bring, where it left most threads idle)
    const int64_t nl = every ? 0 : min(nx, n);
    const int64_t stride = (int64_t)blocks * B;
    unsigned long long cs = 0, ch = 0;
    if (every && blockIdx.x == 0 && threadIdx.x == 0) {
        cs = (unsigned long long)nnz;
        ch = (unsigned long long)hub_cols;
    }
    int64_t t = blockIdx.x * (int64_t)B + threadIdx.x;
    for (; t + 3 * stride < nl; t += 4 * stride) {
        int32_t j[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) j[q] = __ldg(xidx + t + q * stride);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int32_t d = __ldg(colptr + j[q] + 1) - __ldg(colptr + j[q]);
            cs += (unsigned long long)d;
            ch += d > kLongSeg;
        }
    }
    for (; t < nl; t += stride) {
        const int32_t j = __ldg(xidx + t);
        const int32_t d = __ldg(colptr + j + 1) - __ldg(colptr + j);
        cs += (unsigned long long)d;
        ch += d > kLongSeg;
    }
    // the order check: four indices per 16-byte load (where the list is
    // 16-byte aligned), four loads per thread in flight, counting entries t
    // whose column is not t
    unsigned long long cm = 0;
    if (ident) {
        const int64_t gt = blockIdx.x * (int64_t)B + threadIdx.x;
        int64_t q0 = 0;
        if (((uintptr_t)xidx & 15) == 0) {
            const int64_t n4 = n / 4;
            const int4* __restrict__ xv = reinterpret_cast<const int4*>(xidx);
            int64_t q = gt;
            for (; q + 3 * stride < n4; q += 4 * stride) {
                int4 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = __ldg(xv + q + u * stride);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int32_t j = (int32_t)(4 * (q + u * stride));
                    cm += (v[u].x != j) + (v[u].y != j + 1) + (v[u].z != j + 2) + (v[u].w != j + 3);
                }
            }
            for (; q < n4; q += stride) {
                const int4 v = __ldg(xv + q);
                const int32_t j = (int32_t)(4 * q);
                cm += (v.x != j) + (v.y != j + 1) + (v.z != j + 2) + (v.w != j + 3);
            }
            q0 = 4 * n4;
        }
        for (int64_t q = q0 + gt; q < n; q += stride) cm += __ldg(xidx + q) != (int32_t)q;
    }
    finish_counts<B>(blockIdx.x == 0 && threadIdx.x == 0 ? (unsigned long long)nx : 0ull, cs, ch, counters, ticket,
                     desc, di, n, nnz, status, sa, blocks, sn, nq, ident, cm);
}

// Few blocks per SM: every block of the feature pass ends with atomics on
// the same counters and ticket, so thousands of blocks would serialise there.
static int feat_grid(asv_matrix_s* H, int64_t items) {
    const int64_t g = (items + 255) / 256;
    return (int)max((int64_t)1, min(g, (int64_t)H->num_sms * 4));
}

template <class T>
static void* feat_dense_func() {
    return (void*)k_feat_dense<T, 256>;
}

// Fills the launch of this call's feature pass (function, grid, argument
// values and the pointer array), for a direct launch or for updating the
// feature node of the selector-driven graph.
void feature_launch(asv_matrix_s* H, const DescInit& di, const SelectArg& sa, FeatLaunch& fl) {
    fl.di = di;
    fl.sa = sa;
    fl.colptr = H->colptr;
    fl.counters = H->ws.counters;
    fl.ticket = H->ws.ticket;
    fl.desc = H->d_desc;
    fl.n = H->n;
    fl.nnz = H->nnz;
    fl.status = H->ws.status;
    fl.block = dim3(256);
    if (!di.x_sparse) {
        switch (H->dtype) {
            case ASV_F32: fl.func = feat_dense_func<float>(); break;
            case ASV_F64: fl.func = feat_dense_func<double>(); break;
            case ASV_I32: fl.func = feat_dense_func<int32_t>(); break;
            default: fl.func = feat_dense_func<bool8>(); break;
        }
        const int64_t nsuper = (H->n + 127) / 128;
        // six blocks per SM (the kernel's registers leave room for six): the
        // pass streams x with one 16-byte load per lane and step, so the
        // number of warps in flight sets its bandwidth
        fl.grid = dim3((unsigned)max((int64_t)1, min((nsuper + 7) / 8, (int64_t)H->num_sms * 6)));
        fl.xptr = di.user_x_dense;
        fl.xbits = H->ws.xbits_dense;
        void* a[11] = {&fl.xptr, &fl.n, &fl.colptr, &fl.xbits, &fl.counters, &fl.ticket, &fl.desc, &fl.di,
                       &fl.nnz, &fl.status, &fl.sa};
        for (int i = 0; i < 11; ++i) fl.args[i] = a[i];
    } else {
        fl.func = (void*)k_feat_sparse<256>;
        fl.grid = dim3((unsigned)feat_grid(H, H->n));
        fl.nnz_x_dev = di.user_nnz_x;
        fl.xidx = di.user_xidx;
        fl.hub_cols = H->hub_cols;
        void* a[12] = {&fl.nnz_x_dev, &fl.xidx, &fl.colptr, &fl.counters, &fl.ticket, &fl.desc, &fl.di,
                       &fl.n, &fl.nnz, &fl.status, &fl.sa, &fl.hub_cols};
        for (int i = 0; i < 12; ++i) fl.args[i] = a[i];
    }
}

void launch_features(asv_matrix_s* H, const DescInit& di, const SelectArg& sa, cudaStream_t s) {
    FeatLaunch fl;
    feature_launch(H, di, sa, fl);
    cudaLaunchKernel(fl.func, fl.grid, fl.block, fl.args, 0, s);
}

// ---------------------------------------------------------------- sparse x -> dense x + bitmap
// Sets (or clears) x's bit in the scatter bitmap. Lanes of a warp whose
// entries fall into the same 32-bit word (a sorted list puts up to 32 of
// them there) combine their bits first, so each word takes one atomic per
// warp instead of one per entry.
__device__ __forceinline__ void scatter_bit(uint32_t* xbits, int32_t j, bool set) {
    const uint32_t w = (uint32_t)j >> 5;
    if (!set) {
        xbits[w] = 0u;
        return;
    }
    const unsigned peers = __match_any_sync(__activemask(), w);
    const uint32_t word = __reduce_or_sync(peers, 1u << (j & 31));
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicOr(&xbits[w], word);
}

// Scatters a listed x into the zero-invariant dense workspace (set) or
// restores it to zero (clear). BITS: also the scatter bitmap, which only the
// kernels that validate entries, flag output rows or read Boolean terms use.
// A Boolean x is its bitmap alone: every Boolean kernel reads its terms
// from the bitmap when there is one, so the byte vector is never written.
template <class T, bool BITS>
__global__ void k_x_scatter(const CallDesc* __restrict__ desc, T* xdense, uint32_t* xbits, int set, int64_t n) {
    constexpr bool kDense = !(Sr<T>::kPattern && BITS);
    const int64_t nx = desc->nnz_x;
    const int32_t* __restrict__ xidx = desc->xidx;
    const T* __restrict__ xval = (const T*)desc->xval;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const bool vals = xval && !Sr<T>::kPattern;
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    // a list of every column in order: the pull kernels read its values in
    // place, so only the bitmap is set (every bit below n) or cleared
    if (desc->x_ident) {
        if (BITS) {
            const int64_t full = n >> 5;
            for (int64_t w = t; w < (n + 31) / 32; w += stride)
                xbits[w] = !set ? 0u : (w < full ? 0xffffffffu : ((1u << (n & 31)) - 1u));
        }
        return;
    }
    // a list covering more than a quarter of the columns is cleared by
    // writing the whole workspace (16-byte stores) rather than by reading the
    // list again and scattering zeros
    if (!set && 4 * nx > n) {
        if (kDense) {
            const int64_t nv = (int64_t)((n * sizeof(T)) / 16);
            for (int64_t i = t; i < nv; i += stride) reinterpret_cast<uint4*>(xdense)[i] = make_uint4(0u, 0u, 0u, 0u);
            for (int64_t j = nv * (16 / (int64_t)sizeof(T)) + t; j < n; j += stride) xdense[j] = T(0);
        }
        if (BITS)
            for (int64_t w = t; w < (n + 31) / 32; w += stride) xbits[w] = 0u;
        return;
    }
    // four entries per thread in flight (independent index and value loads)
    for (; t + 3 * stride < nx; t += 4 * stride) {
        int32_t j[4];
        T v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            j[q] = xidx[t + q * stride];
            v[q] = (set && vals) ? xval[t + q * stride] : (set ? Sr<T>::one() : T(0));
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (kDense) xdense[j[q]] = v[q];
            if (BITS) scatter_bit(xbits, j[q], set);
        }
    }
    for (; t < nx; t += stride) {
        const int32_t j = xidx[t];
        if (kDense) xdense[j] = set ? (vals ? xval[t] : Sr<T>::one()) : T(0);
        if (BITS) scatter_bit(xbits, j, set);
    }
}

template <class T>
static void x_scatter_dtype(asv_matrix_s* H, bool set, bool bits, int g, cudaStream_t s) {
    if (bits) k_x_scatter<T, true><<<g, 256, 0, s>>>(H->d_desc, (T*)H->ws.xdense, H->ws.xbits_scat, set, H->n);
    else k_x_scatter<T, false><<<g, 256, 0, s>>>(H->d_desc, (T*)H->ws.xdense, H->ws.xbits_scat, set, H->n);
}

void launch_x_scatter(asv_matrix_s* H, bool set, bool bits, cudaStream_t s) {
    const int g = feat_grid(H, H->n);
    switch (H->dtype) {
        case ASV_F32: x_scatter_dtype<float>(H, set, bits, g, s); break;
        case ASV_F64: x_scatter_dtype<double>(H, set, bits, g, s); break;
        case ASV_I32: x_scatter_dtype<int32_t>(H, set, bits, g, s); break;
        case ASV_BOOL: x_scatter_dtype<bool8>(H, set, true, g, s); break;
    }
}

// ---------------------------------------------------------------- ordered compaction
// Over a bitmap (32 items per word) or a byte-flag array (4 items per
// 32-bit word). Block b owns a contiguous word range; a block scan of the
// words' item counts plus the block's offset gives every set item its
// ascending output position.
template <bool BYTES>
__device__ __forceinline__ uint32_t item_mask(uint32_t w) {
    if constexpr (BYTES) {
        // bit 8q+7 set iff byte q is nonzero
        return (((w & 0x7f7f7f7fu) + 0x7f7f7f7fu) | w) & 0x80808080u;
    } else {
        return w;
    }
}

template <bool BYTES>
__device__ __forceinline__ void load_run(const uint32_t* __restrict__ words, int64_t w0, int64_t hi, bool vec,
                                         uint32_t (&m)[kRun]) {
    if (vec && w0 + kRun <= hi) {
        const uint4 a = *reinterpret_cast<const uint4*>(words + w0);
        const uint4 b = *reinterpret_cast<const uint4*>(words + w0 + 4);
        m[0] = a.x; m[1] = a.y; m[2] = a.z; m[3] = a.w;
        m[4] = b.x; m[5] = b.y; m[6] = b.z; m[7] = b.w;
    } else {
#pragma unroll
        for (int q = 0; q < kRun; ++q) m[q] = w0 + q < hi ? words[w0 + q] : 0u;
    }
#pragma unroll
    for (int q = 0; q < kRun; ++q) m[q] = item_mask<BYTES>(m[q]);
}

// Items of each block's range, one run of kRun words (two 16-byte loads) per
// thread and round.
template <int B, bool BYTES>
__global__ void __launch_bounds__(B) k_items_count(const uint32_t* __restrict__ words, int64_t nwords, int32_t* blk,
                                                   Gate gate, CompactSkip skip) {
    if (gate.off() || skip.on()) return;
    __shared__ int32_t sm[B / 32 + 1];
    int64_t lo, hi;
    block_range(nwords, lo, hi);
    const bool vec = ((uintptr_t)words & 15) == 0;
    int32_t s = 0;
    for (int64_t w0 = lo + (int64_t)threadIdx.x * kRun; w0 < hi; w0 += (int64_t)B * kRun) {
        uint32_t m[kRun];
        load_run<BYTES>(words, w0, hi, vec, m);
#pragma unroll
        for (int q = 0; q < kRun; ++q) s += __popc(m[q]);
    }
    s = block_reduce_sum<B>(s, sm);
    if (threadIdx.x == 0) blk[blockIdx.x] = s;
}

// Per round a thread takes a run of consecutive words (kRun byte-flag words,
// or one bitmap word -- at most 32 items either way), all its loads issued
// before the round's one block scan. The items' indices are staged in shared
// memory at their offsets within the round and written out by consecutive
// threads to consecutive output positions, so the stores of a warp are
// contiguous rather than one scattered word per thread.
template <int B, bool BYTES, class Policy>
__global__ void __launch_bounds__(B) k_items_write(uint32_t* words, int64_t nwords, const int32_t* __restrict__ blk,
                                                   Policy pol, Gate gate) {
    if (gate.off()) return;
    constexpr int RUN = BYTES ? kRun : 1;  // words per thread and round
    constexpr int CAP = B * 32;            // items per round at most
    __shared__ int32_t sm[B / 32 + 1];
    // slot k lives at k + k / 32: a thread writes its items to consecutive
    // slots, so with every thread holding 32 items (a dense set) the lanes
    // of a warp would otherwise all hit one bank at each step
    __shared__ int32_t stage[CAP + CAP / 32];
    int64_t lo, hi;
    block_range(nwords, lo, hi);
    if (pol.bypass()) {
        pol.write_bypass(words, lo, hi);
        return;
    }
    const bool vec = ((uintptr_t)words & 15) == 0;
    int32_t base = block_prefix<B>(blk, blockIdx.x, sm);  // blk holds the raw block counts
    pol.begin();
    for (int64_t off = lo; off < hi; off += (int64_t)B * RUN) {
        const int64_t w0 = off + (int64_t)threadIdx.x * RUN;
        uint32_t m[kRun];
        if constexpr (BYTES) {
            load_run<BYTES>(words, w0, hi, vec, m);
        } else {
            m[0] = w0 < hi ? words[w0] : 0u;
        }
        int32_t c = 0;
#pragma unroll
        for (int q = 0; q < RUN; ++q) c += __popc(m[q]);
        int32_t tot;
        int32_t p = block_excl_scan<B>(c, sm, &tot);
#pragma unroll
        for (int q = 0; q < RUN; ++q) {
            uint32_t mask = m[q];
            if (!mask) continue;
            const int64_t w = w0 + q;
            pol.clear_word(words, w);
            while (mask) {
                const int b = __ffs(mask) - 1;
                mask &= mask - 1;
                stage[p + (p >> 5)] = (int32_t)(BYTES ? w * 4 + (b >> 3) : w * 32 + b);
                ++p;
            }
        }
        __syncthreads();
        // four items per thread in flight: every source value of a group is
        // loaded before any of the group's outputs is stored (a store can
        // alias the next source load, so the compiler would not reorder them)
        for (int32_t k0 = threadIdx.x; k0 < tot; k0 += 4 * B) {
            int32_t j[4];
            typename Policy::V v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int32_t k = k0 + u * B;
                j[u] = k < tot ? stage[k + (k >> 5)] : 0;
                if (k < tot) v[u] = pol.load(j[u]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int32_t k = k0 + u * B;
                if (k < tot) pol.store(base + k, j[u], v[u]);
            }
        }
        __syncthreads();
        base += tot;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) pol.count(base);
}

// An output policy of the compaction: load(j) reads item j's value, store()
// writes item j at output position pos.
// dense x -> ascending list (values gathered from x)
template <class T>
struct XListPolicy {
    using V = T;
    const CallDesc* desc;
    int32_t* idx;
    T* val;
    const T* x;
    int64_t bits_below;  // > 0: a list shorter than this is not built (the warp push reads the bitmap)
    __device__ void begin() { x = (const T*)desc->x_dense; }
    __device__ bool bypass() const { return bits_below > 0 && desc->nnz_x < bits_below; }
    __device__ void write_bypass(uint32_t*, int64_t, int64_t) {}
    __device__ void clear_word(uint32_t*, int64_t) {}
    __device__ T load(int32_t j) const { return Sr<T>::kPattern ? Sr<T>::one() : x[j]; }
    __device__ void store(int32_t pos, int32_t j, T v) const {
        idx[pos] = j;
        if (!Sr<T>::kPattern) val[pos] = v;
    }
    __device__ void count(int32_t) {}
};

// public dense -> sparse conversion
template <class T>
struct PublicCompactPolicy {
    using V = T;
    const T* x;
    int32_t* idx;
    T* val;
    int64_t* count_out;
    __device__ void begin() {}
    __device__ bool bypass() const { return false; }
    __device__ void write_bypass(uint32_t*, int64_t, int64_t) {}
    __device__ void clear_word(uint32_t*, int64_t) {}
    __device__ T load(int32_t j) const { return val ? x[j] : T(0); }
    __device__ void store(int32_t pos, int32_t j, T v) const {
        idx[pos] = j;
        if (val) val[pos] = v;
    }
    __device__ void count(int32_t c) { *count_out = c; }
};

// The push accumulator of a row as a value: an A (the value type's Atom, or
// the value type itself for the FP32 accumulators of short-row matrices).
template <class T, class A>
__device__ __forceinline__ T acc_value(A a) {
    if constexpr (std::is_same<A, T>::value) return a;
    else return Sr<T>::from_atom(a);
}

// structural output set -> (yidx, yval, nnz_y); the source is the push
// accumulators of type A (re-zeroed as they are read) or the pull kernels'
// dense y.
template <class T, bool FROM_ACC, class A = typename Sr<T>::Atom>
struct OutSparsePolicy {
    using V = T;
    const CallDesc* desc;
    A* acc;
    const T* ywork;
    int32_t* status;
    int32_t* yidx;
    T* yval;
    int64_t cap;
    int64_t m;  // rows of the output (the flags' items)
    __device__ void begin() {
        yidx = desc->yidx;
        yval = (T*)desc->yval;
        cap = desc->y_cap;
    }
    // every row is in the set (y_ident): the pull wrote the values in place,
    // so this block clears its range of flag words and writes the indices
    // of its rows; block 0 publishes the count m
    __device__ bool bypass() const { return !FROM_ACC && desc->y_ident; }
    __device__ void write_bypass(uint32_t* words, int64_t lo, int64_t hi) const {
        int32_t* __restrict__ yi = desc->yidx;
        for (int64_t w = lo + threadIdx.x; w < hi; w += blockDim.x) words[w] = 0u;
        const int64_t e = min(4 * hi, m);
        for (int64_t i = 4 * lo + threadIdx.x; i < e; i += blockDim.x) yi[i] = (int32_t)i;
        if (blockIdx.x == 0 && threadIdx.x == 0) *desc->nnz_y = m;
    }
    __device__ void clear_word(uint32_t* bits, int64_t w) { bits[w] = 0u; }
    __device__ T load(int32_t i) const {
        if (Sr<T>::kPattern) return Sr<T>::one();
        if (FROM_ACC) return acc_value<T, A>(acc[i]);
        return ywork[i];
    }
    __device__ void store(int32_t pos, int32_t i, T v) const {
        if (FROM_ACC && !Sr<T>::kPattern) acc[i] = A(0);
        if (pos < cap) {
            yidx[pos] = i;
            if (yval) yval[pos] = v;
        }
    }
    __device__ void count(int32_t c) {
        *desc->nnz_y = c;
        if (c > cap) latch_status(status, ASV_ERR_CAPACITY);
    }
};

template <bool BYTES, class Policy>
static void compact_items(asv_matrix_s* H, uint32_t* words, int64_t nitems, const Policy& pol, cudaStream_t s,
                          CompactSkip skip = CompactSkip{}) {
    const int64_t nwords = BYTES ? (nitems + 3) / 4 : (nitems + 31) / 32;
    const int G = H->G;
    const Gate gate = gate_of(H);
    k_items_count<256, BYTES><<<G, 256, 0, s>>>(words, nwords, H->ws.blk, gate, skip);
    k_items_write<256, BYTES, Policy><<<G, 256, 0, s>>>(words, nwords, H->ws.blk, pol, gate);
}

template <class T>
static void x_list_dtype(asv_matrix_s* H, cudaStream_t s, int64_t bits_below) {
    XListPolicy<T> pol{H->d_desc, H->ws.xlist_idx, (T*)H->ws.xlist_val, nullptr, bits_below};
    compact_items<false>(H, H->ws.xbits_dense, H->n, pol, s,
                         CompactSkip{nullptr, bits_below > 0 ? &H->d_desc->nnz_x : nullptr, bits_below});
}

void launch_x_compact_list(asv_matrix_s* H, cudaStream_t s, int64_t bits_below) {
    switch (H->dtype) {
        case ASV_F32: x_list_dtype<float>(H, s, bits_below); break;
        case ASV_F64: x_list_dtype<double>(H, s, bits_below); break;
        case ASV_I32: x_list_dtype<int32_t>(H, s, bits_below); break;
        case ASV_BOOL: x_list_dtype<bool8>(H, s, bits_below); break;
    }
}

// ---------------------------------------------------------------- dense write-out of the push accumulators
// y_i = the accumulator of a flagged row (re-zeroed, its flag cleared) or 0.
// A warp takes 512 rows per step: its lanes load the rows' flags with one
// 16-byte load each (the flag array is padded to a multiple of 16 bytes),
// stage them in shared memory, and then handle the rows 32 at a time with
// consecutive lanes on consecutive rows, so every accumulator load and
// every y store of a warp is one contiguous run. A group of 512 rows without
// a flag (most of them for a sparse product) only writes zeros.
constexpr int kFinRows = 512;
template <class T, class A = typename Sr<T>::Atom>
__global__ void __launch_bounds__(256) k_finalize_dense(int64_t m, A* acc, uint8_t* yflag,
                                                        const CallDesc* __restrict__ desc, Gate gate) {
    if (gate.off()) return;
    using S = Sr<T>;
    __shared__ __align__(16) uint8_t s_f[8][kFinRows];
    T* __restrict__ y = (T*)desc->y;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t ngroups = (m + kFinRows - 1) / kFinRows;
    const int64_t nw = (int64_t)gridDim.x * 8;
    for (int64_t g = (int64_t)blockIdx.x * 8 + w; g < ngroups; g += nw) {
        const int64_t i0 = g * kFinRows;
        const uint4 fw = *reinterpret_cast<const uint4*>(yflag + i0 + 16 * lane);
        *reinterpret_cast<uint4*>(&s_f[w][16 * lane]) = fw;
        const bool any = __any_sync(0xffffffffu, (fw.x | fw.y | fw.z | fw.w) != 0u);
        __syncwarp();
        if (any) *reinterpret_cast<uint4*>(yflag + i0 + 16 * lane) = make_uint4(0u, 0u, 0u, 0u);
        // sixteen rows per lane in flight: loads first, then the stores
        T v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int64_t i = i0 + 32 * u + lane;
            const bool f = any && s_f[w][32 * u + lane] != 0;
            if (S::kPattern) v[u] = f ? S::one() : T(0);
            else v[u] = f ? acc_value<T, A>(acc[i]) : T(0);
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int64_t i = i0 + 32 * u + lane;
            if (i >= m) break;
            y[i] = v[u];
            if constexpr (!S::kPattern) {
                if (any && s_f[w][32 * u + lane]) acc[i] = A(0);
            }
        }
        __syncwarp();
    }
}

template <class T, class Atom>
static void finalize_acc(asv_matrix_s* H, bool from_acc, int out_mode, cudaStream_t s) {
    if (out_mode == ASV_OUT_DENSE) {
        if (H->m > 0) {
            const int64_t groups = (H->m + kFinRows - 1) / kFinRows;
            const int64_t g = std::min<int64_t>((groups + 7) / 8, (int64_t)H->num_sms * 8);
            k_finalize_dense<T, Atom><<<(unsigned)g, 256, 0, s>>>(H->m, (Atom*)H->ws.acc, H->ws.yflag, H->d_desc,
                                                                 gate_of(H));
        }
    } else if (from_acc) {
        OutSparsePolicy<T, true, Atom> pol{H->d_desc, (Atom*)H->ws.acc, nullptr, H->ws.status, nullptr, nullptr, 0};
        compact_items<true>(H, (uint32_t*)H->ws.yflag, H->m, pol, s);
    } else {
        OutSparsePolicy<T, false> pol{H->d_desc, nullptr, (const T*)H->ws.ywork, H->ws.status, nullptr, nullptr, 0,
                                      H->m};
        compact_items<true>(H, (uint32_t*)H->ws.yflag, H->m, pol, s, CompactSkip{&H->d_desc->y_ident, nullptr, 0});
    }
}

// narrow: the push accumulated in FP32 (FP32 matrices with short rows only)
void launch_finalize(asv_matrix_s* H, bool from_acc, int out_mode, cudaStream_t s, bool narrow) {
    switch (H->dtype) {
        case ASV_F32:
            if (narrow) finalize_acc<float, float>(H, from_acc, out_mode, s);
            else finalize_acc<float, typename Sr<float>::Atom>(H, from_acc, out_mode, s);
            break;
        case ASV_F64: finalize_acc<double, typename Sr<double>::Atom>(H, from_acc, out_mode, s); break;
        case ASV_I32: finalize_acc<int32_t, typename Sr<int32_t>::Atom>(H, from_acc, out_mode, s); break;
        case ASV_BOOL: finalize_acc<bool8, typename Sr<bool8>::Atom>(H, from_acc, out_mode, s); break;
    }
}

// ---------------------------------------------------------------- public dense -> sparse
template <class T>
__global__ void k_x_bits(const T* __restrict__ x, int64_t n, uint32_t* xbits) {
    const int lane = threadIdx.x & 31;
    const int64_t nwords = (n + 31) >> 5;
    for (int64_t w = blockIdx.x * (int64_t)(blockDim.x / 32) + (threadIdx.x >> 5); w < nwords;
         w += (int64_t)gridDim.x * (blockDim.x / 32)) {
        const int64_t j = w * 32 + lane;
        const bool nz = j < n && Sr<T>::nz(x[j]);
        const unsigned b = __ballot_sync(0xffffffffu, nz);
        if (lane == 0) xbits[w] = b;
    }
}

template <class T>
static void compact_public_dtype(asv_matrix_s* H, const void* x, int32_t* idx, void* val, int64_t* count,
                                 cudaStream_t s) {
    const int g = feat_grid(H, ((H->n + 31) / 32) * 32);
    k_x_bits<T><<<g, 256, 0, s>>>((const T*)x, H->n, H->ws.xbits_dense);
    PublicCompactPolicy<T> pol{(const T*)x, idx, (T*)val, count};
    compact_items<false>(H, H->ws.xbits_dense, H->n, pol, s);
}

void launch_compact_public(asv_matrix_s* H, const void* x, int32_t* idx, void* val, int64_t* count, cudaStream_t s) {
    switch (H->dtype) {
        case ASV_F32: compact_public_dtype<float>(H, x, idx, val, count, s); break;
        case ASV_F64: compact_public_dtype<double>(H, x, idx, val, count, s); break;
        case ASV_I32: compact_public_dtype<int32_t>(H, x, idx, val, count, s); break;
        case ASV_BOOL: compact_public_dtype<bool8>(H, x, idx, val, count, s); break;
    }
}

}  // namespace asv
