// Batched products Y[b,:] = A x_b for B sparse vectors in one captured,
// persistent launch (an extension of the paper's single-vector method), and
// the batched backward pass of y = A x (dx = A^T dy, dA on A's pattern).
//
// Forward. The batch arrives as a CSR of vectors (xptr[B+1], xidx, xval) or
// dense [B][n]. It is first regrouped by column -- a stable radix sort of
// the entries by column id, so that each column's list of (vector id, value)
// is ascending in the vector id -- and then a persistent kernel pulls work
// items (a tile of R consecutive rows of A) x (a group of GB vectors) from an
// atomic queue. Warp w owns row i0+w of the tile: for every entry (j, a) of
// that row it walks the part of column j's list that falls in the vector
// group and adds a*x_b[j] into a shared-memory tile acc[w][b] of
// compensated (Neumaier) sums, one (sum, correction) float pair per output
// (row stride GB+1 pairs, so that the lanes of one step, which hold
// ascending vector ids, touch consecutive 8-byte words). An output can sum
// hundreds of products (the longest rows against the longest vectors of a
// Zipf batch), so a plain FP32 sum would not keep the 2e-6 relative bound.
// Lanes of one step hold distinct vector ids and a warp's columns are taken
// in order, so the accumulation needs no atomics and is deterministic. Each column of A
// is read once per vector group instead of once per vector, and every
// element of Y is written exactly once, with R consecutive values per vector.
//
// Hot columns. When a few columns of A are shared by most vectors of the
// batch (Zipf-distributed features: the 128 most popular columns of the
// 1M x 131k benchmark matrix carry 98 % of the batch's multiply-adds), the
// product restricted to those columns is a dense one: the batch's entries in
// the hot columns are scattered into a dense [H][B] block Xh (zeros where a
// vector lacks the column), and a persistent kernel gives each thread one
// vector and each work item R rows: the item's slice of Xh sits in shared
// memory, the rows' hot entries (in row order) are read as broadcasts, and
// every thread sums its R outputs with fused multiply-adds in registers --
// groups of eight terms in FP32, groups added with compensation -- and
// writes them, so the kernel writes all of Y. The remaining (cold) entries
// of the batch are then pushed through A's CSC view with FP32 atomic adds
// into Y. Hot columns are those present in at least theta vectors, theta
// the smallest power of two that keeps their number within H (chosen on
// the device from a histogram of the columns' batch counts).
//
// Backward. With dY and X given dense [B][m] and [B][n]: both are
// transposed to vector-minor layouts (dYt[m][B], Xt[n][B]) so that one
// matrix entry meets B contiguous values; dX^T[j][:] = sum over column j of
// a_ij dYt[i][:] reads the CSC once for the whole batch, and
// dA_k = <dYt[row(k)][:], Xt[col(k)][:]> reads the CSR once.
#include "internal.h"
#include "prims.cuh"
#include "sort.cuh"

namespace asv {

// Per-call pointers of a batched product, read by every kernel of the
// captured pipeline (the graph's kernel arguments stay fixed).
struct BatchDesc {
    const int64_t* xptr;   // CSR of vectors (NULL when X is dense)
    const int32_t* xidx;
    const float* xval;     // NULL = all ones
    const float* Xdense;   // [B][n] or NULL
    float* Y;              // [B][m]
    int64_t cap;           // workspace capacity in entries
};

// ---------------------------------------------------------------- batch regrouping
// The entry count, clamped to the workspace (a larger batch latches an error).
__global__ void k_batch_count(const BatchDesc* __restrict__ bd, int32_t B, int64_t* wptr, int64_t* count,
                              int32_t* status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (bd->Xdense) return;  // the dense path fills wptr itself
    int64_t e = bd->xptr[B] - bd->xptr[0];
    if (e > bd->cap) {
        latch_status(status, ASV_ERR_CAPACITY);
        e = bd->cap;
    }
    *count = e;
}

// entry e of vector b -> (key = column, payload = b << 32 | value bits)
__global__ void k_batch_pack(const BatchDesc* __restrict__ bd, int32_t B, const int64_t* __restrict__ count,
                             uint32_t* keys, uint64_t* pay) {
    if (bd->Xdense) return;
    const int64_t* xptr = bd->xptr;
    const int64_t base = xptr[0], cnt = *count;
    for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
        const int64_t lo = xptr[b] - base, hi = min(xptr[b + 1] - base, cnt);
        for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
            keys[e] = (uint32_t)bd->xidx[e + base];
            const float v = bd->xval ? bd->xval[e + base] : 1.0f;
            pay[e] = ((uint64_t)(uint32_t)b << 32) | (uint64_t)__float_as_uint(v);
        }
    }
}

// dense [B][n]: per-vector nonzero counts, an exclusive scan, then the entries
__global__ void k_dense_count(const BatchDesc* __restrict__ bd, int32_t B, int64_t n, int64_t* cnt) {
    __shared__ unsigned long long sm[8 + 1];
    const float* X = bd->Xdense;
    if (!X) return;
    for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
        unsigned long long c = 0;
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) c += X[b * n + j] != 0.0f;
        c = block_reduce_sum<256>(c, sm);
        if (threadIdx.x == 0) cnt[b + 1] = (int64_t)c;
    }
}

__global__ void k_dense_scan(const BatchDesc* __restrict__ bd, int64_t* cnt, int32_t B, int64_t* count) {
    if (!bd->Xdense || threadIdx.x != 0 || blockIdx.x != 0) return;
    cnt[0] = 0;
    for (int32_t b = 0; b < B; ++b) cnt[b + 1] += cnt[b];
    *count = cnt[B];
}

__global__ void k_dense_emit(const BatchDesc* __restrict__ bd, int32_t B, int64_t n, const int64_t* __restrict__ xptr,
                             uint32_t* keys, uint64_t* pay) {
    __shared__ int32_t sm[8 + 1];
    const float* X = bd->Xdense;
    if (!X) return;
    for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
        int32_t base = (int32_t)xptr[b];
        for (int64_t off = 0; off < n; off += 256) {
            const int64_t j = off + threadIdx.x;
            const float v = j < n ? X[b * n + j] : 0.0f;
            const int32_t f = v != 0.0f;
            int32_t tot;
            const int32_t pos = base + block_excl_scan<256>(f, sm, &tot);
            if (f) {
                keys[pos] = (uint32_t)j;
                pay[pos] = ((uint64_t)(uint32_t)b << 32) | (uint64_t)__float_as_uint(v);
            }
            base += tot;
        }
    }
}

// column pointers of the regrouped batch (count on the device)
__global__ void k_batch_colptr(const uint32_t* __restrict__ key, const int64_t* __restrict__ count, int64_t n,
                               int32_t* cptr) {
    const int64_t E = *count;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p <= E; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t prev = p == 0 ? -1 : (int64_t)key[p - 1];
        const int64_t cur = p == E ? n : (int64_t)key[p];
        for (int64_t c = prev + 1; c <= cur; ++c) cptr[c] = (int32_t)p;
    }
}

// ---------------------------------------------------------------- forward kernel
// first position in [lo, hi) of a column list whose vector id is >= b0
__device__ __forceinline__ int32_t lower_b(const uint64_t* __restrict__ pay, int32_t lo, int32_t hi, uint32_t b0) {
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if ((uint32_t)(pay[mid] >> 32) < b0) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <int R>
__global__ void __launch_bounds__(R * 32) k_batched_fwd(const BatchDesc* __restrict__ bd, int64_t m, int32_t B,
                                                        int32_t GB, const int32_t* __restrict__ rowptr,
                                                        const int32_t* __restrict__ col, const float* __restrict__ val,
                                                        const int32_t* __restrict__ cptr,
                                                        const uint64_t* __restrict__ pay, unsigned long long* queue,
                                                        unsigned int* ticket) {
    extern __shared__ float2 acc[];  // [R][GB + 1] of (sum, correction)
    __shared__ long long s_item;
    __shared__ bool s_last;
    float* __restrict__ Y = bd->Y;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t ntiles = (m + R - 1) / R;
    const int32_t ngroups = (B + GB - 1) / GB;
    const long long total = (long long)ntiles * ngroups;
    while (true) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(queue, 1ull);
        __syncthreads();
        const long long item = s_item;
        if (item >= total) break;
        const int64_t tile = item / ngroups;
        const int32_t g = (int32_t)(item % ngroups);
        const uint32_t b0 = (uint32_t)g * GB;
        const int32_t nb = min(GB, B - (int32_t)b0);
        const int GBp = GB + 1;
        for (int e = threadIdx.x; e < GBp * R; e += blockDim.x) acc[e] = make_float2(0.0f, 0.0f);
        __syncthreads();
        const int64_t i = tile * R + w;
        if (i < m) {
            const int32_t rb = __ldg(rowptr + i), re = __ldg(rowptr + i + 1);
            for (int32_t k = rb; k < re; ++k) {
                const int32_t j = __ldg(col + k);
                const float a = val ? __ldg(val + k) : 1.0f;
                int32_t lo = __ldg(cptr + j), hi = __ldg(cptr + j + 1);
                if (ngroups > 1) {
                    lo = lower_b(pay, lo, hi, b0);
                    hi = lower_b(pay, lo, hi, b0 + (uint32_t)nb);
                }
                for (int32_t q = lo + lane; q < hi; q += 32) {
                    const uint64_t pv = __ldg(pay + q);
                    const uint32_t b = (uint32_t)(pv >> 32) - b0;
                    KahanF k;
                    const float2 cur = acc[w * GBp + b];
                    k.s = cur.x;
                    k.c = cur.y;
                    k.add(__fmul_rn(a, __uint_as_float((uint32_t)pv)));
                    acc[w * GBp + b] = make_float2(k.s, k.c);
                }
                __syncwarp();
            }
        }
        __syncthreads();
        // write the tile: vector b gets R consecutive values of its row of Y
        const int64_t r0 = tile * R;
        const int rr = (int)min((int64_t)R, m - r0);
        for (int e = threadIdx.x; e < nb * R; e += blockDim.x) {
            const int b = e / R, r = e % R;
            if (r < rr) {
                const float2 sc = acc[r * GBp + b];
                Y[(int64_t)(b0 + b) * m + r0 + r] = __fadd_rn(sc.x, sc.y);
            }
        }
        __syncthreads();
    }
    // the last block out resets the queue (zero-invariant)
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        atomicExch(queue, 0ull);
        __threadfence();
        atomicExch(ticket, 0u);
    }
}

// ---------------------------------------------------------------- hot-column path
constexpr int kHotMinCount = 16;  // a column shared by fewer vectors stays cold

// histogram of the columns' batch counts by bit length (bin b: counts in [2^(b-1), 2^b))
__global__ void k_hot_hist(const int32_t* __restrict__ cptr, int64_t n, int32_t* hist) {
    __shared__ int32_t sh[33];
    for (int i = threadIdx.x; i < 33; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = cptr[j + 1] - cptr[j];
        if (c >= kHotMinCount) atomicAdd(&sh[32 - __clz(c)], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 33; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// theta = the smallest power of two whose columns (counts >= theta) number
// at most hmax; the histogram is re-zeroed for the next call
__global__ void k_hot_pick(int32_t* hist, int32_t hmax, int32_t* theta, int32_t* hot_n) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int32_t acc = 0, th = 0x7fffffff;
    for (int b = 32; b >= 1; --b) {
        if (acc + hist[b] > hmax) break;
        acc += hist[b];
        if (hist[b] > 0 || acc > 0) th = 1 << (b - 1);
    }
    *theta = max(th, kHotMinCount);
    *hot_n = 0;
    for (int b = 0; b < 33; ++b) hist[b] = 0;
}

__global__ void k_hot_assign(const int32_t* __restrict__ cptr, int64_t n, const int32_t* __restrict__ theta,
                             int32_t* hot_id, int32_t* hot_n) {
    const int32_t th = *theta;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = cptr[j + 1] - cptr[j];
        hot_id[j] = c >= th ? atomicAdd(hot_n, 1) : -1;
    }
}

// the batch's entries in hot columns -> Xh[h][b]
__global__ void k_hot_scatter(const uint32_t* __restrict__ key, const uint64_t* __restrict__ pay,
                              const int64_t* __restrict__ count, const int32_t* __restrict__ hot_id, int32_t B,
                              float* Xh) {
    const int64_t E = *count;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t h = hot_id[key[e]];
        if (h >= 0) {
            const uint64_t pv = pay[e];
            Xh[(int64_t)h * B + (uint32_t)(pv >> 32)] = __uint_as_float((uint32_t)pv);
        }
    }
}

// A's entries split once per call into per-row lists, in row order: hot
// entries (slot, a) and the cold entries (j, a) whose column some vector of
// the batch holds; entries in columns no vector holds are dropped.
__global__ void k_split_count(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, int64_t m,
                              const int32_t* __restrict__ hot_id, const int32_t* __restrict__ cptr, int32_t* hcnt,
                              int32_t* ccnt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t h = 0, c = 0;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            const int32_t j = __ldg(col + k);
            if (__ldg(hot_id + j) >= 0) ++h;
            else if (__ldg(cptr + j + 1) > __ldg(cptr + j)) ++c;
        }
        hcnt[i] = h;
        ccnt[i] = c;
    }
}

__global__ void k_split_fill(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const float* __restrict__ val, int64_t m, const int32_t* __restrict__ hot_id,
                             const int32_t* __restrict__ cptr, const int32_t* __restrict__ hrow,
                             const int32_t* __restrict__ crow, int2* hent, int2* cent) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t ph = hrow[i], pc = crow[i];
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            const int32_t j = __ldg(col + k);
            const float a = val ? __ldg(val + k) : 1.0f;
            const int32_t h = __ldg(hot_id + j);
            if (h >= 0) hent[ph++] = make_int2(h, __float_as_int(a));
            else if (__ldg(cptr + j + 1) > __ldg(cptr + j)) cent[pc++] = make_int2(j, __float_as_int(a));
        }
    }
}

// For every cold column j that some vector holds: tb[j*(nvt+1) + t] = first
// position of its (vector-ascending) list whose vector is in tile t or later.
__global__ void k_tile_bounds(const int32_t* __restrict__ cptr, const uint64_t* __restrict__ pay, int64_t n,
                              const int32_t* __restrict__ hot_id, int32_t nvt, int32_t V, int32_t* tb) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t lo = cptr[j], hi = cptr[j + 1];
        if (hi <= lo || hot_id[j] >= 0) continue;
        int32_t* t = tb + j * (int64_t)(nvt + 1);
        int32_t p = lo;
        for (int32_t u = 0; u <= nvt; ++u) {
            const uint32_t first_b = (uint32_t)u * (uint32_t)V;
            while (p < hi && (uint32_t)(pay[p] >> 32) < first_b) ++p;
            t[u] = p;
        }
    }
}

template <int R, int V, int HM>
__global__ void __launch_bounds__(V) k_batched_hot(const BatchDesc* __restrict__ bd, int64_t m, int32_t B,
                                                  const int32_t* __restrict__ hrow, const int2* __restrict__ hent,
                                                  const int32_t* __restrict__ crow, const int2* __restrict__ cent,
                                                  const int32_t* __restrict__ tb, const uint64_t* __restrict__ pay,
                                                  const int32_t* __restrict__ hot_n, const float* __restrict__ Xh,
                                                  unsigned long long* queue, unsigned int* ticket) {
    __shared__ int2 s_ent[R * HM];                // the item's hot entries: (slot * B, a), rows in order
    __shared__ float s_cold[R][V + 1];            // cold contributions of the item, then its outputs
    __shared__ int32_t s_hrow[R + 1], s_crow[R + 1];
    __shared__ long long s_item;
    __shared__ bool s_last;
    float* __restrict__ Y = bd->Y;
    const int32_t H = min(*hot_n, HM);
    const int64_t ntiles = (m + R - 1) / R;
    const int32_t nvt = (B + V - 1) / V;
    const long long total = (long long)ntiles * nvt;
    while (true) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(queue, 1ull);
        __syncthreads();
        const long long item = s_item;
        if (item >= total) break;
        const int32_t vt = (int32_t)(item / ntiles);   // vector-tile major: the grid shares one slice
        const int64_t r0 = (item % ntiles) * R;
        const int nr = (int)min((int64_t)R, m - r0);
        const int32_t b0 = vt * V;
        const int32_t b = b0 + (int32_t)threadIdx.x;
        if (threadIdx.x <= R) {
            const int64_t i = r0 + min((int)threadIdx.x, nr);
            s_hrow[threadIdx.x] = __ldg(hrow + i);
            s_crow[threadIdx.x] = __ldg(crow + i);
        }
        for (int e = threadIdx.x; e < R * (V + 1); e += V) (&s_cold[0][0])[e] = 0.0f;
        __syncthreads();
        // the item's hot entries (contiguous: its rows are consecutive)
        const int32_t h0 = s_hrow[0], hn = min(s_hrow[nr] - h0, R * HM);
        for (int e = threadIdx.x; e < hn; e += V) {
            const int2 en = __ldg(hent + h0 + e);
            s_ent[e] = make_int2(en.x * B, en.y);
        }
        // cold entries: each thread takes entries of the item's rows and adds
        // a * x_b for the vectors b of this tile that hold the column
        const int32_t c0 = s_crow[0], cn = s_crow[nr] - c0;
        for (int e = threadIdx.x; e < cn; e += V) {
            const int2 en = __ldg(cent + c0 + e);
            int r = 0;
            while (r + 1 < nr && s_crow[r + 1] <= c0 + e) ++r;
            const int32_t* t = tb + (int64_t)en.x * (nvt + 1) + vt;
            const int32_t lo = __ldg(t), hi = __ldg(t + 1);
            for (int32_t q = lo; q < hi; ++q) {
                const uint64_t pv = __ldg(pay + q);
                atomicAdd(&s_cold[r][(int32_t)(pv >> 32) - b0],
                          __fmul_rn(__int_as_float(en.y), __uint_as_float((uint32_t)pv)));
            }
        }
        __syncthreads();
        if (b < B) {
            // the tile's slice of Xh (H rows of V floats) stays in L1: every
            // block of the grid works on the same vector tile at a time
            const float* __restrict__ xt = Xh + b;
            for (int r = 0; r < nr; ++r) {
                KahanF acc;
                acc.zero();
                const int qb = s_hrow[r] - h0, qe = min(s_hrow[r + 1] - h0, R * HM);
                int q = qb;
                for (; q + 8 <= qe; q += 8) {
                    float p = 0.0f;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int2 en = s_ent[q + u];  // one broadcast read per term
                        p = __fmaf_rn(__int_as_float(en.y), __ldg(xt + en.x), p);
                    }
                    acc.add(p);
                }
                float p = 0.0f;
                for (; q < qe; ++q) {
                    const int2 en = s_ent[q];
                    p = __fmaf_rn(__int_as_float(en.y), __ldg(xt + en.x), p);
                }
                acc.add(p);
                acc.add(s_cold[r][threadIdx.x]);
                s_cold[r][threadIdx.x] = acc.value();  // only this thread reads (r, tid)
            }
        }
        __syncthreads();
        // write-out: a warp instruction covers 32 / R vectors' runs of R
        // consecutive rows (whole 32-byte sectors of Y), not 32 scattered words
        {
            constexpr int VPI = 32 / R;  // vectors per instruction
            const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
            const int r = lane % R;
            for (int it = 0; it < R; ++it) {
                const int v = w * 32 + it * VPI + lane / R;
                const int32_t bv = b0 + v;
                if (bv < B && r < nr) Y[(int64_t)bv * m + r0 + r] = s_cold[r][v];
            }
        }
        __syncthreads();
    }
    // the last block out resets the queue (zero-invariant)
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        atomicExch(queue, 0ull);
        __threadfence();
        atomicExch(ticket, 0u);
    }
}

// ---------------------------------------------------------------- backward kernels
// out[c][r] = in[r][c] for a rows x cols FP32 matrix (32x32 shared tiles)
__global__ void k_transpose(const float* __restrict__ in, float* __restrict__ out, int64_t rows, int64_t cols) {
    __shared__ float t[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = r0 + k, c = c0 + threadIdx.x;
        if (r < rows && c < cols) t[k][threadIdx.x] = in[r * cols + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t c = c0 + k, r = r0 + threadIdx.x;
        if (c < cols && r < rows) out[c * rows + r] = t[threadIdx.x][k];
    }
}

// dXt[j][:] = sum_{k in column j} a_k * dYt[rowidx_k][:]; one warp per column,
// lane l holds vectors l, l+32, ... (B <= 128).
template <int VPL>
__global__ void __launch_bounds__(256) k_bwd_dx(int64_t n, int32_t B, const int32_t* __restrict__ colptr,
                                                const int32_t* __restrict__ rowidx, const float* __restrict__ valc,
                                                const float* __restrict__ dYt, float* __restrict__ dXt) {
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (j >= n) return;
    KahanF acc[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v) acc[v].zero();
    const int32_t b = __ldg(colptr + j), e = __ldg(colptr + j + 1);
    for (int32_t k = b; k < e; ++k) {
        const float a = valc ? __ldg(valc + k) : 1.0f;
        const float* src = dYt + (int64_t)__ldg(rowidx + k) * B;
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            const int bb = lane + 32 * v;
            if (bb < B) acc[v].add(__fmul_rn(a, __ldg(src + bb)));
        }
    }
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int bb = lane + 32 * v;
        if (bb < B) dXt[j * B + bb] = acc[v].value();
    }
}

// dA_k = sum_b dYt[i][b] * Xt[col_k][b] for the entries of row i; one warp
// per row, the warp's lanes split the vectors and reduce with shuffles.
template <int VPL>
__global__ void __launch_bounds__(256) k_bwd_da(int64_t m, int32_t B, const int32_t* __restrict__ rowptr,
                                                const int32_t* __restrict__ col, const float* __restrict__ dYt,
                                                const float* __restrict__ Xt, float* __restrict__ dA) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i >= m) return;
    float dy[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int bb = lane + 32 * v;
        dy[v] = bb < B ? __ldg(dYt + i * B + bb) : 0.0f;
    }
    const int32_t b = __ldg(rowptr + i), e = __ldg(rowptr + i + 1);
    for (int32_t k = b; k < e; ++k) {
        const float* xs = Xt + (int64_t)__ldg(col + k) * B;
        float s = 0.0f;
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            const int bb = lane + 32 * v;
            if (bb < B) s = __fadd_rn(s, __fmul_rn(dy[v], __ldg(xs + bb)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s = __fadd_rn(s, __shfl_xor_sync(0xffffffffu, s, o));
        if (lane == 0) dA[k] = s;
    }
}

// ---------------------------------------------------------------- host side
static int bitlen(int64_t v) {
    int b = 0;
    while (v > 0) { ++b; v >>= 1; }
    return b;
}

static void bfree(void*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

// Batch workspaces grow on demand (a call that needs more memory allocates
// and synchronises; steady-state calls allocate nothing).
static cudaError_t batch_workspace(asv_matrix_s* H, int64_t entries, int32_t B) {
    BatchWs& bw = H->bws;
    cudaError_t e;
    if (!bw.desc) {
        if ((e = cudaMalloc(&bw.desc, sizeof(BatchDesc))) != cudaSuccess) return e;
        if ((e = cudaMalloc((void**)&bw.queue, 64)) != cudaSuccess) return e;
        if ((e = cudaMemset(bw.queue, 0, 64)) != cudaSuccess) return e;
        if ((e = cudaMalloc((void**)&bw.cptr, 4 * (H->n + 1))) != cudaSuccess) return e;
    }
    if (entries > bw.cap_entries || B > bw.cap_B) {
        void* ps[5] = {bw.keys[0], bw.keys[1], bw.pay[0], bw.pay[1], bw.xptr};
        cudaDeviceSynchronize();
        for (void* p : ps) if (p) cudaFree(p);
        const int64_t E = std::max<int64_t>(entries, 1024);
        const int32_t BB = std::max<int32_t>(B, 64);
        if ((e = cudaMalloc((void**)&bw.keys[0], 4 * E)) != cudaSuccess) return e;
        if ((e = cudaMalloc((void**)&bw.keys[1], 4 * E)) != cudaSuccess) return e;
        if ((e = cudaMalloc((void**)&bw.pay[0], 8 * E)) != cudaSuccess) return e;
        if ((e = cudaMalloc((void**)&bw.pay[1], 8 * E)) != cudaSuccess) return e;
        if ((e = cudaMalloc((void**)&bw.xptr, 8 * (BB + 2))) != cudaSuccess) return e;
        bw.cap_entries = E;
        bw.cap_B = BB;
        for (auto& kv : bw.graphs) {
            cudaGraphExecDestroy(kv.second);
        }
        bw.graphs.clear();
    }
    return cudaSuccess;
}

static void fwd_kernel(asv_matrix_s* H, int32_t B, int R, int GB, const uint64_t* pay, cudaStream_t s) {
    BatchWs& bw = H->bws;
    const size_t shm = (size_t)R * (GB + 1) * sizeof(float2);
    int per_sm = 1;
    unsigned long long* q = (unsigned long long*)bw.queue;
    unsigned int* tk = (unsigned int*)(bw.queue + 1);
    const float* val = (const float*)H->val;
    const BatchDesc* bd = (const BatchDesc*)bw.desc;
#define FWD(RR)                                                                                                 \
    do {                                                                                                        \
        cudaFuncSetAttribute(k_batched_fwd<RR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);         \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched_fwd<RR>, RR * 32, shm);               \
        const int grid = H->num_sms * std::max(per_sm, 1);                                                      \
        k_batched_fwd<RR><<<grid, RR * 32, shm, s>>>(bd, H->m, B, GB, H->rowptr, H->col, val, bw.cptr, pay, q, tk); \
    } while (0)
    switch (R) {
        case 4: FWD(4); break;
        case 8: FWD(8); break;
        default: FWD(16); break;
    }
#undef FWD
}

static cudaError_t hot_workspace(asv_matrix_s* H, int32_t hot, int32_t V) {
    BatchWs& bw = H->bws;
    cudaError_t e;
    bool moved = false;
    if (!bw.hot_id) {
        const int64_t m1 = H->m + 1, nnz = std::max<int64_t>(H->nnz, 1);
        if ((e = cudaMalloc((void**)&bw.hot_id, 4 * std::max<int64_t>(H->n, 1))) != cudaSuccess) return e;
        if ((e = cudaMalloc((void**)&bw.hot_ctl, 4 * 40)) != cudaSuccess) return e;
        if ((e = cudaMemset(bw.hot_ctl, 0, 4 * 40)) != cudaSuccess) return e;
        if ((e = cudaMalloc((void**)&bw.hrow, 4 * (m1 + 1))) != cudaSuccess) return e;
        if ((e = cudaMalloc((void**)&bw.crow, 4 * (m1 + 1))) != cudaSuccess) return e;
        if ((e = cudaMalloc((void**)&bw.hent, 8 * nnz)) != cudaSuccess) return e;
        if ((e = cudaMalloc((void**)&bw.cent, 8 * nnz)) != cudaSuccess) return e;
    }
    const int64_t need = (int64_t)hot * bw.cap_B;
    if (need > bw.xh_cap) {
        cudaDeviceSynchronize();
        bfree(bw.xh);
        if ((e = cudaMalloc(&bw.xh, 4 * need)) != cudaSuccess) return e;
        bw.xh_cap = need;
        moved = true;
    }
    const int64_t tneed = std::max<int64_t>(H->n, 1) * ((bw.cap_B + V - 1) / V + 1);
    if (tneed > bw.tb_cap) {
        cudaDeviceSynchronize();
        bfree(bw.tb);
        if ((e = cudaMalloc(&bw.tb, 4 * tneed)) != cudaSuccess) return e;
        bw.tb_cap = tneed;
        moved = true;
    }
    if (moved) {  // captured pipelines hold the old buffers
        for (auto& kv : bw.graphs) cudaGraphExecDestroy(kv.second);
        bw.graphs.clear();
    }
    return cudaSuccess;
}

// hot columns -> dense Xh; A split into per-row hot and cold lists; the cold
// columns' tile bounds; the persistent kernel that writes Y
static void hot_pipeline(asv_matrix_s* H, int32_t B, int R, int V, int hot, const uint32_t* key,
                         const uint64_t* pay, const int64_t* count, cudaStream_t s) {
    BatchWs& bw = H->bws;
    int32_t* hist = bw.hot_ctl;          // [33]
    int32_t* theta = bw.hot_ctl + 33;
    int32_t* hot_n = bw.hot_ctl + 34;
    const int g = H->num_sms * 4;
    k_hot_hist<<<g, 256, 0, s>>>(bw.cptr, H->n, hist);
    k_hot_pick<<<1, 32, 0, s>>>(hist, hot, theta, hot_n);
    k_hot_assign<<<g, 256, 0, s>>>(bw.cptr, H->n, theta, bw.hot_id, hot_n);
    cudaMemsetAsync(bw.xh, 0, 4 * (size_t)hot * B, s);
    k_hot_scatter<<<g, 256, 0, s>>>(key, pay, count, bw.hot_id, B, (float*)bw.xh);
    const float* val = (const float*)H->val;
    k_split_count<<<H->num_sms * 8, 256, 0, s>>>(H->rowptr, H->col, H->m, bw.hot_id, bw.cptr, bw.hrow, bw.crow);
    scan_excl(bw.hrow, bw.hrow, H->m, nullptr, H->ws.blk, H->G, true, s);
    scan_excl(bw.crow, bw.crow, H->m, nullptr, H->ws.blk, H->G, true, s);
    k_split_fill<<<H->num_sms * 8, 256, 0, s>>>(H->rowptr, H->col, val, H->m, bw.hot_id, bw.cptr, bw.hrow, bw.crow,
                                                (int2*)bw.hent, (int2*)bw.cent);
    const int32_t nvt = (B + V - 1) / V;
    k_tile_bounds<<<g, 256, 0, s>>>(bw.cptr, pay, H->n, bw.hot_id, nvt, V, (int32_t*)bw.tb);
    unsigned long long* q = (unsigned long long*)bw.queue;
    unsigned int* tk = (unsigned int*)(bw.queue + 1);
    const BatchDesc* bd = (const BatchDesc*)bw.desc;
#define HOT(RR, VV, HH)                                                                                        \
    do {                                                                                                       \
        int per_sm = 1;                                                                                        \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched_hot<RR, VV, HH>, VV, 0);             \
        const int grid = H->num_sms * std::max(per_sm, 1);                                                     \
        k_batched_hot<RR, VV, HH><<<grid, VV, 0, s>>>(bd, H->m, B, bw.hrow, (const int2*)bw.hent, bw.crow,     \
                                                        (const int2*)bw.cent, (const int32_t*)bw.tb, pay, hot_n, \
                                                        (const float*)bw.xh, q, tk);                           \
    } while (0)
    if (hot <= 64) {
        if (R <= 8) { if (V <= 128) HOT(8, 128, 64); else HOT(8, 256, 64); }
        else { if (V <= 128) HOT(16, 128, 64); else HOT(16, 256, 64); }
    } else {
        if (R <= 8) { if (V <= 128) HOT(8, 128, 128); else HOT(8, 256, 128); }
        else { if (V <= 128) HOT(16, 128, 128); else HOT(16, 256, 128); }
    }
#undef HOT
}

// The batched pipeline: entry count, regrouping by column (radix sort), column
// pointers, then the persistent forward kernel (or the hot-column pipeline).
static void enqueue_batched(asv_matrix_s* H, int32_t B, int R, int GB, int hot, cudaStream_t s) {
    BatchWs& bw = H->bws;
    const BatchDesc* bd = (const BatchDesc*)bw.desc;
    int64_t* count = bw.xptr + (bw.cap_B + 1);
    const int gb = (int)std::min<int64_t>(B, 4096);
    k_batch_count<<<1, 32, 0, s>>>(bd, B, bw.xptr, count, H->ws.status);
    k_dense_count<<<gb, 256, 0, s>>>(bd, B, H->n, bw.xptr);
    k_dense_scan<<<1, 32, 0, s>>>(bd, bw.xptr, B, count);
    k_dense_emit<<<gb, 256, 0, s>>>(bd, B, H->n, bw.xptr, bw.keys[0], bw.pay[0]);
    k_batch_pack<<<gb, 128, 0, s>>>(bd, B, count, bw.keys[0], bw.pay[0]);
    uint32_t* kb[2] = {bw.keys[0], bw.keys[1]};
    uint64_t* vb[2] = {bw.pay[0], bw.pay[1]};
    const int cur = radix_sort<uint64_t, true>(kb, vb, 0, count, bitlen(H->n - 1), H->ws.hist, H->ws.blk, H->G, s);
    k_batch_colptr<<<H->num_sms * 8, 256, 0, s>>>(kb[cur], count, H->n, bw.cptr);
    if (hot > 0) hot_pipeline(H, B, R, GB, hot, kb[cur], vb[cur], count, s);
    else fwd_kernel(H, B, R, GB, vb[cur], s);
}

cudaError_t batched_forward(asv_matrix_s* H, int32_t B, int64_t max_entries, const int64_t* xptr, const int32_t* xidx,
                            const float* xval, const float* Xdense, float* Y, int R, int GB, int hot,
                            cudaStream_t s) {
    const int64_t need = Xdense ? (int64_t)B * H->n : max_entries;
    cudaError_t e = batch_workspace(H, need, B);
    if (e != cudaSuccess) return e;
    if (hot > 0 && (e = hot_workspace(H, hot, GB)) != cudaSuccess) return e;
    BatchWs& bw = H->bws;
    BatchDesc hd{xptr, xidx, xval, Xdense, Y, bw.cap_entries};
    if ((e = cudaMemcpyAsync(bw.desc, &hd, sizeof(hd), cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
    const long long key = ((long long)B << 24) | ((long long)hot << 16) | ((long long)R << 12) | (long long)GB;
    auto it = bw.graphs.find(key);
    if (it == bw.graphs.end()) {
        if (!H->cap_stream) {
            if ((e = cudaStreamCreateWithFlags(&H->cap_stream, cudaStreamNonBlocking)) != cudaSuccess) return e;
        }
        cudaGraph_t g;
        if ((e = cudaStreamBeginCapture(H->cap_stream, cudaStreamCaptureModeRelaxed)) != cudaSuccess) return e;
        enqueue_batched(H, B, R, GB, hot, H->cap_stream);
        if ((e = cudaStreamEndCapture(H->cap_stream, &g)) != cudaSuccess) return e;
        cudaGraphExec_t ex;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return e;
        it = bw.graphs.emplace(key, ex).first;
    }
    if ((e = cudaGraphLaunch(it->second, s)) != cudaSuccess) return e;
    return cudaGetLastError();
}

// ---------------------------------------------------------------- backward
static cudaError_t bwd_workspace(asv_matrix_s* H, int32_t B) {
    BatchWs& bw = H->bws;
    if (B <= bw.bwd_B) return cudaSuccess;
    cudaDeviceSynchronize();
    bfree(bw.dYt);
    bfree(bw.Xt);
    bfree(bw.dXt);
    cudaError_t e;
    if ((e = cudaMalloc(&bw.dYt, 4 * (size_t)B * std::max<int64_t>(H->m, 1))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&bw.Xt, 4 * (size_t)B * std::max<int64_t>(H->n, 1))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&bw.dXt, 4 * (size_t)B * std::max<int64_t>(H->n, 1))) != cudaSuccess) return e;
    bw.bwd_B = B;
    return cudaSuccess;
}

static void transpose(const float* in, float* out, int64_t rows, int64_t cols, cudaStream_t s) {
    if (rows == 0 || cols == 0) return;
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    k_transpose<<<grid, dim3(32, 8), 0, s>>>(in, out, rows, cols);
}

// A listed batch (CSR of vectors) into the vector-minor dense layout Xt[n][B]
// that the dA kernel reads (zeroed before): block b writes vector b's
// entries; a column id outside [0, n) is skipped and reported.
__global__ void k_list_to_xt(const int64_t* __restrict__ xptr, const int32_t* __restrict__ xidx,
                             const float* __restrict__ xval, int64_t n, int32_t B, float* Xt, int32_t* status) {
    const int32_t b = blockIdx.x;
    const int64_t base = xptr[0];
    const int64_t lo = xptr[b] - base, hi = xptr[b + 1] - base;
    for (int64_t t = lo + threadIdx.x; t < hi; t += blockDim.x) {
        const int32_t j = xidx[t];
        if ((uint64_t)(uint32_t)j >= (uint64_t)n) {
            latch_status(status, ASV_ERR_ARG);
            continue;
        }
        Xt[(int64_t)j * B + b] = xval ? xval[t] : 1.0f;
    }
}

cudaError_t batched_backward(asv_matrix_s* H, int32_t B, const float* X, const float* dY, float* dX, float* dA,
                             cudaStream_t s, const int64_t* xptr, const int32_t* xidx, const float* xval) {
    cudaError_t e = bwd_workspace(H, B);
    if (e != cudaSuccess) return e;
    BatchWs& bw = H->bws;
    float* dYt = (float*)bw.dYt;
    float* Xt = (float*)bw.Xt;
    float* dXt = (float*)bw.dXt;
    transpose(dY, dYt, B, H->m, s);
    const int vpl = (B + 31) / 32;
    if (dX && H->n > 0) {
        const unsigned g = (unsigned)((H->n + 7) / 8);
        const float* vc = (const float*)H->val_csc;
        switch (vpl) {
            case 1: k_bwd_dx<1><<<g, 256, 0, s>>>(H->n, B, H->colptr, H->rowidx, vc, dYt, dXt); break;
            case 2: k_bwd_dx<2><<<g, 256, 0, s>>>(H->n, B, H->colptr, H->rowidx, vc, dYt, dXt); break;
            case 3: k_bwd_dx<3><<<g, 256, 0, s>>>(H->n, B, H->colptr, H->rowidx, vc, dYt, dXt); break;
            default: k_bwd_dx<4><<<g, 256, 0, s>>>(H->n, B, H->colptr, H->rowidx, vc, dYt, dXt); break;
        }
        transpose(dXt, dX, H->n, B, s);
    }
    if (dA && H->m > 0 && H->nnz > 0) {
        if (xptr) {  // listed x: conversion to the layout the kernel reads (Sec. VI-A online conversion)
            cudaMemsetAsync(Xt, 0, 4 * (size_t)B * H->n, s);
            k_list_to_xt<<<B, 256, 0, s>>>(xptr, xidx, xval, H->n, B, Xt, H->ws.status);
        } else {
            transpose(X, Xt, B, H->n, s);
        }
        const unsigned g = (unsigned)((H->m + 7) / 8);
        switch (vpl) {
            case 1: k_bwd_da<1><<<g, 256, 0, s>>>(H->m, B, H->rowptr, H->col, dYt, Xt, dA); break;
            case 2: k_bwd_da<2><<<g, 256, 0, s>>>(H->m, B, H->rowptr, H->col, dYt, Xt, dA); break;
            case 3: k_bwd_da<3><<<g, 256, 0, s>>>(H->m, B, H->rowptr, H->col, dYt, Xt, dA); break;
            default: k_bwd_da<4><<<g, 256, 0, s>>>(H->m, B, H->rowptr, H->col, dYt, Xt, dA); break;
        }
    }
    return cudaGetLastError();
}

void batch_release(asv_matrix_s* H) {
    BatchWs& bw = H->bws;
    for (auto& kv : bw.graphs) cudaGraphExecDestroy(kv.second);
    bw.graphs.clear();
    void* ps[] = {bw.keys[0], bw.keys[1], bw.pay[0], bw.pay[1], bw.xptr, bw.cptr, bw.desc, bw.queue, bw.dYt, bw.Xt,
                  bw.dXt, bw.hot_id, bw.hot_ctl, bw.xh, bw.hrow, bw.crow, bw.hent, bw.cent, bw.tb};
    for (void* p : ps) if (p) cudaFree(p);
}

}  // namespace asv
