// Level bookkeeping of the breadth-first search built on the masked product
// (the BFS application of Sec. VII): the search starts from one vertex, and
// every new frontier -- the ascending list of rows the masked product
// reached -- gets its level and joins the visited set, which masks the next
// product.
#include "internal.h"

namespace asv {

__global__ void k_bfs_init(int32_t source, int32_t* level, uint32_t* visited, int32_t* front, int64_t* count) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    level[source] = 0;
    visited[source >> 5] = 1u << (source & 31);
    front[0] = source;
    count[0] = 1;
    count[1] = 0;
}

// Each vertex of the new frontier appears once (the output list is a set),
// so its level is written by one thread; visited bits share words, hence
// the atomic OR.
__global__ void k_bfs_visit(const int32_t* __restrict__ front, const int64_t* __restrict__ count, int32_t* level,
                            uint32_t* visited, int32_t depth) {
    const int64_t nf = *count;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nf; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = front[t];
        level[v] = depth;
        atomicOr(visited + (v >> 5), 1u << (v & 31));
    }
}

void launch_bfs_init(int32_t source, int32_t* level, uint32_t* visited, int32_t* front, int64_t* count,
                     cudaStream_t s) {
    k_bfs_init<<<1, 32, 0, s>>>(source, level, visited, front, count);
}

void launch_bfs_visit(const int32_t* front, const int64_t* count, int32_t* level, uint32_t* visited, int32_t depth,
                      int grid, cudaStream_t s) {
    k_bfs_visit<<<grid, 256, 0, s>>>(front, count, level, visited, depth);
}

}  // namespace asv

// ---------------------------------------------------------------- incremental PageRank
// Level bookkeeping of the delta-form PageRank driver (the incremental
// PageRank application of Sec. VII): the rank is the sum of the deltas
// delta_{k+1} = d A D^{-1} delta_k, delta_0 = (1 - d)/N; deltas below eps
// are dropped, so the input vector of the product thins out as the
// iteration converges.
namespace asv {

template <class T>
__global__ void k_pr_init(int64_t n, T c, T* rank, int32_t* didx, T* dval, int64_t* count) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        rank[j] = c;
        didx[j] = (int32_t)j;
        dval[j] = c;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        count[0] = n;
        count[1] = 0;
    }
}

// x_j = delta_j / deg(j) over the delta list (0 for a column with no entries)
template <class T>
__global__ void k_pr_scale(const int32_t* __restrict__ didx, const T* __restrict__ dval,
                           const int64_t* __restrict__ count, const int32_t* __restrict__ colptr, T* xval) {
    const int64_t nx = *count;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nx; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j = didx[t];
        const int32_t deg = colptr[j + 1] - colptr[j];
        xval[t] = deg > 0 ? dval[t] / (T)deg : T(0);
    }
}

// delta_i = d y_i for the rows of the product: added to the rank, and kept
// for the next product when |delta_i| >= eps. The output rows are distinct,
// so the rank updates do not collide; the kept list is appended in any order.
template <class T>
__global__ void k_pr_update(const int32_t* __restrict__ yidx, const T* __restrict__ yval,
                            const int64_t* __restrict__ ycount, T damping, T eps, T* rank, int32_t* didx, T* dval,
                            int64_t* dcount) {
    const int64_t ny = *ycount;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ny; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = yidx[t];
        const T v = damping * yval[t];
        rank[i] += v;
        if (fabs((double)v) >= (double)eps) {
            const int64_t q = (int64_t)atomicAdd((unsigned long long*)dcount, 1ull);
            didx[q] = i;
            dval[q] = v;
        }
    }
}

void launch_pr_init(int32_t dtype, int64_t n, double c, void* rank, int32_t* didx, void* dval, int64_t* count,
                    int grid, cudaStream_t s) {
    if (dtype == ASV_F64)
        k_pr_init<double><<<grid, 256, 0, s>>>(n, c, (double*)rank, didx, (double*)dval, count);
    else
        k_pr_init<float><<<grid, 256, 0, s>>>(n, (float)c, (float*)rank, didx, (float*)dval, count);
}

void launch_pr_scale(int32_t dtype, const int32_t* didx, const void* dval, const int64_t* count,
                     const int32_t* colptr, void* xval, int grid, cudaStream_t s) {
    if (dtype == ASV_F64)
        k_pr_scale<double><<<grid, 256, 0, s>>>(didx, (const double*)dval, count, colptr, (double*)xval);
    else
        k_pr_scale<float><<<grid, 256, 0, s>>>(didx, (const float*)dval, count, colptr, (float*)xval);
}

void launch_pr_update(int32_t dtype, const int32_t* yidx, const void* yval, const int64_t* ycount, double damping,
                      double eps, void* rank, int32_t* didx, void* dval, int64_t* dcount, int grid, cudaStream_t s) {
    if (dtype == ASV_F64)
        k_pr_update<double><<<grid, 256, 0, s>>>(yidx, (const double*)yval, ycount, damping, eps, (double*)rank,
                                                 didx, (double*)dval, dcount);
    else
        k_pr_update<float><<<grid, 256, 0, s>>>(yidx, (const float*)yval, ycount, (float)damping, (float)eps,
                                                (float*)rank, didx, (float*)dval, dcount);
}

}  // namespace asv
