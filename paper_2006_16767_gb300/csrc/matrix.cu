// Once-per-matrix work of the runtime procedure (Sec. VI-A, VI-C): the CSC
// view and CSC->CSR map, the Table 1 matrix features, the nnz-balanced
// (merge-path) tile partition of the pull pattern, and optional validation.
#include "internal.h"
#include "prims.cuh"
#include "sort.cuh"

namespace asv {

size_t vsize(int32_t dtype) {
    switch (dtype) {
        case ASV_F32: return 4;
        case ASV_F64: return 8;
        case ASV_I32: return 4;
        case ASV_BOOL: return 1;
    }
    return 0;
}

void scan_excl(const int32_t* in, int32_t* out, int64_t n_h, const int64_t* n_d, int32_t* blk, int G,
               bool write_total, cudaStream_t s) {
    k_scan_reduce<256><<<G, 256, 0, s>>>(in, n_h, n_d, blk);
    k_scan_down<256><<<G, 256, 0, s>>>(in, out, n_h, n_d, blk, write_total ? 1 : 0);
}

// ---------------------------------------------------------------- transpose
__global__ void k_iota(uint32_t* v, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = (uint32_t)i;
}

// row_of[k] = row containing CSR position k; one warp per row.
__global__ void k_expand_rows(const int32_t* rowptr, int64_t m, int32_t* row_of) {
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x >> 5;
    for (int64_t i = blockIdx.x * wpb + (threadIdx.x >> 5); i < m; i += (int64_t)gridDim.x * wpb) {
        const int32_t b = rowptr[i], e = rowptr[i + 1];
        for (int32_t k = b + lane; k < e; k += 32) row_of[k] = (int32_t)i;
    }
}

// colptr from column-sorted keys: position p starts every column in (key[p-1], key[p]].
__global__ void k_colptr_from_sorted(const uint32_t* key, int64_t nnz, int64_t n, int32_t* colptr) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p <= nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t prev = p == 0 ? -1 : (int64_t)key[p - 1];
        const int64_t cur = p == nnz ? n : (int64_t)key[p];
        for (int64_t c = prev + 1; c <= cur; ++c) colptr[c] = (int32_t)p;
    }
}

template <class V>
__global__ void k_gather_csc(const uint32_t* perm, const int32_t* row_of, const V* val, int64_t nnz,
                             int32_t* rowidx, V* val_csc, int32_t* perm_out) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = perm[p];
        perm_out[p] = (int32_t)k;
        rowidx[p] = row_of[k];
        if (val) val_csc[p] = val[k];
    }
}

static int bitlen(int64_t v) {
    int b = 0;
    while (v > 0) { ++b; v >>= 1; }
    return b;
}

cudaError_t build_csc(asv_matrix_s* H, cudaStream_t s) {
    const int64_t nnz = H->nnz;
    const int G = H->G;
    const int grid = H->num_sms * 8;
    if (nnz == 0) {
        cudaMemsetAsync(H->colptr, 0, sizeof(int32_t) * (H->n + 1), s);
        return cudaGetLastError();
    }
    uint32_t *k0 = nullptr, *k1 = nullptr, *v0 = nullptr, *v1 = nullptr;
    int32_t* row_of = nullptr;
    cudaError_t e;
    if ((e = cudaMallocAsync((void**)&k0, 4 * nnz, s)) != cudaSuccess) return e;
    if ((e = cudaMallocAsync((void**)&k1, 4 * nnz, s)) != cudaSuccess) return e;
    if ((e = cudaMallocAsync((void**)&v0, 4 * nnz, s)) != cudaSuccess) return e;
    if ((e = cudaMallocAsync((void**)&v1, 4 * nnz, s)) != cudaSuccess) return e;
    if ((e = cudaMallocAsync((void**)&row_of, 4 * nnz, s)) != cudaSuccess) return e;
    cudaMemcpyAsync(k0, H->col, 4 * nnz, cudaMemcpyDeviceToDevice, s);
    k_iota<<<grid, 256, 0, s>>>(v0, nnz);
    uint32_t* kb[2] = {k0, k1};
    uint32_t* vb[2] = {v0, v1};
    const int cur = radix_sort<uint32_t, true>(kb, vb, nnz, nullptr, bitlen(H->n - 1), H->ws.hist, H->ws.blk, G, s);
    k_expand_rows<<<grid, 256, 0, s>>>(H->rowptr, H->m, row_of);
    k_colptr_from_sorted<<<grid, 256, 0, s>>>(kb[cur], nnz, H->n, H->colptr);
    switch (vsize(H->dtype)) {
        case 8:
            k_gather_csc<<<grid, 256, 0, s>>>(vb[cur], row_of, (const double*)H->val, nnz, H->rowidx,
                                              (double*)H->val_csc, H->perm);
            break;
        case 4:
            k_gather_csc<<<grid, 256, 0, s>>>(vb[cur], row_of, (const uint32_t*)H->val, nnz, H->rowidx,
                                              (uint32_t*)H->val_csc, H->perm);
            break;
        default:
            k_gather_csc<<<grid, 256, 0, s>>>(vb[cur], row_of, (const uint8_t*)nullptr, nnz, H->rowidx,
                                              (uint8_t*)nullptr, H->perm);
    }
    cudaFreeAsync(k0, s);
    cudaFreeAsync(k1, s);
    cudaFreeAsync(v0, s);
    cudaFreeAsync(v1, s);
    cudaFreeAsync(row_of, s);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- features (Table 1)
struct RowStats {
    long long max_row, min_row;
    unsigned long long sum, sumsq;
};

__global__ void k_stats_init(RowStats* st) {
    st->max_row = 0;
    st->min_row = 0x7fffffffffffffffLL;
    st->sum = 0;
    st->sumsq = 0;
}

template <int B>
__global__ void __launch_bounds__(B) k_row_stats(const int32_t* rowptr, int64_t m, RowStats* st) {
    __shared__ unsigned long long sm[B / 32 + 1];
    long long mx = 0, mn = 0x7fffffffffffffffLL;
    unsigned long long s1 = 0, s2 = 0;
    for (int64_t i = blockIdx.x * (int64_t)B + threadIdx.x; i < m; i += (int64_t)gridDim.x * B) {
        const long long d = rowptr[i + 1] - rowptr[i];
        mx = d > mx ? d : mx;
        mn = d < mn ? d : mn;
        s1 += (unsigned long long)d;
        s2 += (unsigned long long)(d * d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        long long a = __shfl_xor_sync(0xffffffffu, mx, o), b = __shfl_xor_sync(0xffffffffu, mn, o);
        mx = a > mx ? a : mx;
        mn = b < mn ? b : mn;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&st->max_row, mx);
        atomicMin(&st->min_row, mn);
    }
    s1 = block_reduce_sum<B>(s1, sm);
    s2 = block_reduce_sum<B>(s2, sm);
    if (threadIdx.x == 0) {
        atomicAdd(&st->sum, s1);
        atomicAdd(&st->sumsq, s2);
    }
}

__global__ void k_degree_hist(const int32_t* rowptr, int64_t m, int32_t* hist) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&hist[rowptr[i + 1] - rowptr[i]], 1);
}

__device__ double i128_to_double(__int128 v) {
    const bool neg = v < 0;
    unsigned __int128 u = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
    const unsigned long long hi = (unsigned long long)(u >> 64), lo = (unsigned long long)u;
    const double r = (double)hi * 18446744073709551616.0 + (double)lo;
    return neg ? -r : r;
}

// Gini numerator over the degree histogram h with exclusive prefix c:
// sorted positions c_d+1 .. c_d+h_d carry weights (2i - m - 1), which sum to
// h_d (2 c_d + h_d - m), so G = sum_d d h_d (2 c_d + h_d - m) / (m nnz).
// Exact in 128-bit integers; finalises every Table 1 matrix feature.
template <int B>
__global__ void __launch_bounds__(B) k_features_final(const int32_t* hist, const int32_t* cum, int64_t maxd,
                                                      int64_t m, int64_t n, const RowStats* st, MatFeat* out) {
    __shared__ __int128 sm[B];
    __int128 acc = 0;
    for (int64_t d = threadIdx.x; d <= maxd; d += B) {
        const __int128 h = hist[d], c = cum[d];
        acc += (__int128)d * h * (2 * c + h - (__int128)m);
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        __int128 num = 0;
        for (int t = 0; t < B; ++t) num += sm[t];
        const long long nnz = (long long)st->sum;
        MatFeat f;
        f.m = m;
        f.n = n;
        f.nnz = nnz;
        f.max_row = m > 0 ? st->max_row : 0;
        f.min_row = m > 0 ? st->min_row : 0;
        f.avg_row = m > 0 ? (double)nnz / (double)m : 0.0;
        f.relative_range = n > 0 ? (double)(f.max_row - f.min_row) / (double)n : 0.0;
        // population variance numerator m*sum(d^2) - (sum d)^2, exact
        const __int128 vn = (__int128)m * (__int128)st->sumsq - (__int128)nnz * (__int128)nnz;
        f.var_nnz_row = m > 0 ? sqrt(i128_to_double(vn) / ((double)m * (double)m)) : 0.0;
        f.gini = (m > 0 && nnz > 0) ? i128_to_double(num) / ((double)m * (double)nnz) : 0.0;
        *out = f;
    }
}

cudaError_t build_features(asv_matrix_s* H, cudaStream_t s) {
    RowStats* st = nullptr;
    cudaError_t e;
    if ((e = cudaMallocAsync((void**)&st, sizeof(RowStats), s)) != cudaSuccess) return e;
    k_stats_init<<<1, 1, 0, s>>>(st);
    if (H->m > 0) k_row_stats<256><<<H->num_sms * 4, 256, 0, s>>>(H->rowptr, H->m, st);
    RowStats hs;
    cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    const int64_t maxd = H->m > 0 ? hs.max_row : 0;
    int32_t *hist = nullptr, *cum = nullptr;
    if ((e = cudaMallocAsync((void**)&hist, 4 * (maxd + 2), s)) != cudaSuccess) return e;
    if ((e = cudaMallocAsync((void**)&cum, 4 * (maxd + 2), s)) != cudaSuccess) return e;
    cudaMemsetAsync(hist, 0, 4 * (maxd + 2), s);
    if (H->m > 0) k_degree_hist<<<H->num_sms * 8, 256, 0, s>>>(H->rowptr, H->m, hist);
    scan_excl(hist, cum, maxd + 1, nullptr, H->ws.blk, H->G, false, s);
    k_features_final<256><<<1, 256, 0, s>>>(hist, cum, maxd, H->m, H->n, st, H->d_mfeat);
    MatFeat hf;
    cudaMemcpyAsync(&hf, H->d_mfeat, sizeof(hf), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(hist, s);
    cudaFreeAsync(cum, s);
    cudaFreeAsync(st, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    H->h_mfeat.m = hf.m;
    H->h_mfeat.n = hf.n;
    H->h_mfeat.nnz = hf.nnz;
    H->h_mfeat.max_row = hf.max_row;
    H->h_mfeat.min_row = hf.min_row;
    H->h_mfeat.avg_row = hf.avg_row;
    H->h_mfeat.relative_range = hf.relative_range;
    H->h_mfeat.var_nnz_row = hf.var_nnz_row;
    H->h_mfeat.gini = hf.gini;
    return cudaGetLastError();
}

// ---------------------------------------------------------------- merge-path partition
// Tile t starts on diagonal t*D of the merge of the row-end offsets
// (rowptr[1..m]) with the nonzero indices 0..nnz-1; tile_row[t] is the number
// of row ends consumed before that diagonal (Merrill & Garland's merge path,
// the load-balanced distribution of Sec. IV-B).
__global__ void k_partition(const int32_t* rowptr, int64_t m, int64_t nnz, int64_t ntiles, int64_t D,
                            int32_t* tile_row) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t <= ntiles; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = min(t * D, m + nnz);
        int64_t lo = max((int64_t)0, d - nnz), hi = min(d, m);
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)rowptr[mid + 1] <= d - mid - 1) lo = mid + 1;
            else hi = mid;
        }
        tile_row[t] = (int32_t)lo;
    }
}

cudaError_t build_partition(asv_matrix_s* H, cudaStream_t s) {
    const int64_t D = pull_tile_items(H->dtype);
    k_partition<<<(int)((H->ntiles + 256) / 256), 256, 0, s>>>(H->rowptr, H->m, H->nnz, H->ntiles, D, H->tile_row);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- long rows
// Counts segments and multi-segment rows of the rows longer than kLongRow.
__global__ void k_long_count(const int32_t* __restrict__ rowptr, int64_t m, unsigned long long* cnt) {
    __shared__ unsigned long long sm[8 + 1];
    unsigned long long ns = 0, nm = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t len = rowptr[i + 1] - rowptr[i];
        if (len > kLongRow) {
            const int32_t k = (len + kLongSeg - 1) / kLongSeg;
            ns += (unsigned long long)k;
            nm += k > 1;
        }
    }
    ns = block_reduce_sum<256>(ns, sm);
    __syncthreads();
    nm = block_reduce_sum<256>(nm, sm);
    if (threadIdx.x == 0) {
        if (ns) atomicAdd(cnt, ns);
        if (nm) atomicAdd(cnt + 1, nm);
    }
}

// Each long row reserves its consecutive run of segment slots with one atomic,
// so a row's segments stay together and in order whatever the slot order.
__global__ void k_long_fill(const int32_t* __restrict__ rowptr, int64_t m, int4* seg, int32_t* multi_row,
                            int32_t* multi_base, unsigned long long* cursor) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t rb = rowptr[i], re = rowptr[i + 1], len = re - rb;
        if (len <= kLongRow) continue;
        const int32_t k = (len + kLongSeg - 1) / kLongSeg;
        const int32_t base = (int32_t)atomicAdd(cursor, (unsigned long long)k);
        for (int32_t t = 0; t < k; ++t) {
            const int32_t b = rb + t * kLongSeg;
            seg[base + t] = make_int4((int32_t)i, b, min(b + kLongSeg, re), k == 1 ? 1 : 0);
        }
        if (k > 1) {
            const int32_t q = (int32_t)atomicAdd(cursor + 1, 1ull);
            multi_row[q] = (int32_t)i;
            multi_base[q] = base;
        }
    }
}

// Columns longer than thr (the hubs of a listed x that covers every column).
__global__ void k_count_over(const int32_t* __restrict__ ptr, int64_t n, int32_t thr, unsigned long long* cnt) {
    unsigned long long c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += ptr[i + 1] - ptr[i] > thr;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

cudaError_t count_hub_columns(asv_matrix_s* H, cudaStream_t s) {
    H->hub_cols = 0;
    if (H->n == 0) return cudaSuccess;
    unsigned long long* d_cnt = (unsigned long long*)H->ws.counters;  // a zeroed word, restored below
    cudaError_t e;
    k_count_over<<<H->num_sms * 8, 256, 0, s>>>(H->colptr, H->n, kLongSeg, d_cnt);
    unsigned long long h = 0;
    if ((e = cudaMemcpyAsync(&h, d_cnt, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(d_cnt, 0, sizeof(h), s)) != cudaSuccess) return e;
    H->hub_cols = (int64_t)h;
    return cudaSuccess;
}

cudaError_t build_long_rows(asv_matrix_s* H, cudaStream_t s) {
    H->nseg = H->nmulti = 0;
    if (H->m == 0 || H->nnz <= kLongRow) return cudaSuccess;
    unsigned long long* d_cnt = (unsigned long long*)H->ws.counters;  // two zeroed words, restored below
    cudaError_t e;
    const int grid = H->num_sms * 8;
    k_long_count<<<grid, 256, 0, s>>>(H->rowptr, H->m, d_cnt);
    unsigned long long h[2] = {0, 0};
    if ((e = cudaMemcpyAsync(h, d_cnt, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(d_cnt, 0, sizeof(h), s)) != cudaSuccess) return e;
    if (h[0] == 0) return cudaSuccess;
    auto grab = [&](void** p, size_t bytes) -> cudaError_t {
        cudaError_t r = cudaMalloc(p, bytes < 16 ? 16 : bytes);
        if (r == cudaSuccess) H->allocs.push_back(*p);
        return r;
    };
    const size_t ns = (size_t)h[0], nm = (size_t)h[1];
    if ((e = grab((void**)&H->seg, 16 * ns)) != cudaSuccess) return e;
    if ((e = grab((void**)&H->long_part, 8 * ns)) != cudaSuccess) return e;
    if ((e = grab((void**)&H->long_hit, ns)) != cudaSuccess) return e;
    if ((e = grab((void**)&H->multi_row, 4 * nm)) != cudaSuccess) return e;
    if ((e = grab((void**)&H->multi_base, 4 * nm)) != cudaSuccess) return e;
    if (H->dtype == ASV_BOOL) {
        // at most (kLongSeg - 256) / 512 + 1 = 8 pieces per segment go to the second pass
        if ((e = grab((void**)&H->long_rest, 16 * 8 * ns)) != cudaSuccess) return e;
        if ((e = grab((void**)&H->long_rest_n, 16)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(H->long_rest_n, 0, 16, s)) != cudaSuccess) return e;
    }
    k_long_fill<<<grid, 256, 0, s>>>(H->rowptr, H->m, H->seg, H->multi_row, H->multi_base, d_cnt);
    if ((e = cudaMemsetAsync(d_cnt, 0, sizeof(h), s)) != cudaSuccess) return e;
    H->nseg = (int64_t)ns;
    H->nmulti = (int64_t)nm;
    return cudaGetLastError();
}

// Tile table of the balanced pull for caller-owned arrays (used by the
// allocation-free entry point).
void launch_partition_raw(const int32_t* rowptr, int64_t m, int64_t nnz, int64_t ntiles, int32_t* tile_row,
                          cudaStream_t s) {
    const int64_t D = pull_tile_items(ASV_F32);
    k_partition<<<(int)((ntiles + 256) / 256), 256, 0, s>>>(rowptr, m, nnz, ntiles, D, tile_row);
}

// ---------------------------------------------------------------- value refresh
template <class V>
__global__ void k_regather(const int32_t* __restrict__ perm, const V* __restrict__ val, int64_t nnz, V* val_csc) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
        val_csc[p] = val[perm[p]];
}

cudaError_t regather_values(asv_matrix_s* H, cudaStream_t s) {
    if (H->nnz == 0 || !H->val || !H->val_csc) return cudaSuccess;
    const int grid = H->num_sms * 8;
    if (vsize(H->dtype) == 8)
        k_regather<<<grid, 256, 0, s>>>(H->perm, (const double*)H->val, H->nnz, (double*)H->val_csc);
    else
        k_regather<<<grid, 256, 0, s>>>(H->perm, (const uint32_t*)H->val, H->nnz, (uint32_t*)H->val_csc);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- transposed view
// The CSC -> CSR position map of A^T: entry p of A's CSC is entry p of A^T's
// CSR and sits at A^T's CSC position perm[p] (A's CSR position).
__global__ void k_invert_perm(const int32_t* __restrict__ perm, int64_t nnz, int32_t* __restrict__ inv) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
        inv[perm[p]] = (int32_t)p;
}

cudaError_t invert_perm(const int32_t* perm, int64_t nnz, int32_t* inv, cudaStream_t s) {
    if (nnz == 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>((nnz + 255) / 256, 4096);  // grid-stride beyond
    k_invert_perm<<<grid, 256, 0, s>>>(perm, nnz, inv);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- validation
__global__ void k_validate(const int32_t* rowptr, const int32_t* col, int64_t m, int64_t n, int64_t nnz,
                           int32_t* flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = rowptr[i], e = rowptr[i + 1];
        if ((i == 0 && b != 0) || (i == m - 1 && e != nnz) || e < b || b < 0 || e > nnz) {
            atomicOr(flag, 1);
            continue;
        }
        for (int64_t k = b; k < e; ++k) {
            const int32_t c = col[k];
            if (c < 0 || c >= n || (k > b && c <= col[k - 1])) {
                atomicOr(flag, 1);
                break;
            }
        }
    }
}

cudaError_t validate_csr(asv_matrix_s* H, cudaStream_t s, int32_t* d_flag) {
    cudaMemsetAsync(d_flag, 0, 4, s);
    if (H->m > 0) k_validate<<<H->num_sms * 8, 256, 0, s>>>(H->rowptr, H->col, H->m, H->n, H->nnz, d_flag);
    return cudaGetLastError();
}

}  // namespace asv
