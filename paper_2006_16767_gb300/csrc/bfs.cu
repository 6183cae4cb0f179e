// Step kernels of the two driver loops built on the selector-driven product
// (the BFS and incremental PageRank applications of Sec. VII). Each loop is
// one CUDA graph: a WHILE node whose body is the product (feature pass,
// selector, chosen candidate) followed by the step kernel here, whose last
// block decides whether another iteration runs -- no host round trip per
// level or iteration.
#include "internal.h"

namespace asv {

// The block that draws the last ticket sees every other block's writes
// (each fences before its ticket) and re-zeroes the ticket for the next step.
__device__ __forceinline__ bool last_block(unsigned int* ticket) {
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        *ticket = 0u;
    }
    return last;
}

// ---------------------------------------------------------------- breadth-first search
// frontier_{d+1} = (A frontier_d) restricted to the unvisited rows: the
// masked product of each level writes the new frontier as an ascending list
// into the `next` list; the step gives those vertices level d, adds them to
// the visited mask and moves the list into the `front` slot the next
// level's product reads.

__global__ void k_bfs_init(int32_t source, int64_t n, int32_t* level, uint32_t* visited, int32_t* front,
                           int64_t* count, LoopState* st) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    level[source] = 0;
    visited[source >> 5] = 1u << (source & 31);
    front[0] = source;
    count[0] = 1;
    count[1] = 0;
    st->out = level;
    st->iter = 1;
    st->max_iter = n;  // a search has at most n - 1 levels after the source's
    st->ticket = 0u;
}

// Each vertex of the new frontier appears once (the output list is a set),
// so its level is written by one thread; visited bits share words, hence
// the atomic OR.
__global__ void k_bfs_step(const int32_t* __restrict__ next, int64_t* count, int32_t* __restrict__ front,
                           uint32_t* visited, LoopState* st, unsigned long long loop) {
    const int64_t nf = count[1];
    const int64_t depth = st->iter;
    int32_t* level = (int32_t*)st->out;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nf; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = next[t];
        level[v] = (int32_t)depth;
        atomicOr(visited + (v >> 5), 1u << (v & 31));
        front[t] = v;
    }
    if (last_block(&st->ticket) && threadIdx.x == 0) {
        count[0] = nf;
        const bool more = nf > 0 && depth < st->max_iter;
        if (more) st->iter = depth + 1;
        cudaGraphSetConditional((cudaGraphConditionalHandle)loop, more ? 1u : 0u);
    }
}

void launch_bfs_init(int32_t source, int64_t n, int32_t* level, uint32_t* visited, int32_t* front, int64_t* count,
                     LoopState* st, cudaStream_t s) {
    k_bfs_init<<<1, 32, 0, s>>>(source, n, level, visited, front, count, st);
}

void launch_bfs_step(const int32_t* next, int64_t* count, int32_t* front, uint32_t* visited, LoopState* st,
                     unsigned long long loop, int grid, cudaStream_t s) {
    k_bfs_step<<<grid, 256, 0, s>>>(next, count, front, visited, st, loop);
}

// ---------------------------------------------------------------- incremental PageRank
// rank = sum of delta_k, delta_0 = (1 - d)/N on every vertex,
// delta_{k+1} = d A D^{-1} delta_k, entries below eps dropped, so the input
// vector of the product thins out as the iteration converges. The product's
// input list holds x_j = delta_j / deg(j) directly: the step that keeps a
// delta also scales it for the next product, in place of the list the
// product has just consumed.

template <class T>
__device__ __forceinline__ T scaled(T delta, const int32_t* __restrict__ colptr, int32_t j) {
    const int32_t deg = colptr[j + 1] - colptr[j];
    return deg > 0 ? delta / (T)deg : T(0);  // a column without entries passes nothing on
}

template <class T>
__global__ void k_pr_init(int64_t n, T c, double damping, double eps, int32_t max_iter, T* rank,
                          const int32_t* __restrict__ colptr, int32_t* xidx, T* xval, int64_t* count, LoopState* st) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        rank[j] = c;
        xidx[j] = (int32_t)j;
        xval[j] = scaled(c, colptr, (int32_t)j);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        count[0] = n;
        count[1] = 0;
        st->out = rank;
        st->iter = 0;
        st->max_iter = max_iter;
        st->p0 = damping;
        st->p1 = eps;
        st->ticket = 0u;
    }
}

// delta_i = d y_i for the rows of the product: added to the rank, and kept
// (scaled) for the next product when |delta_i| >= eps. The output rows are
// distinct, so the rank updates do not collide; the kept list is appended in
// any order at count[1] and becomes the input (count[0]) at the end.
template <class T>
__global__ void k_pr_step(const int32_t* __restrict__ yidx, const T* __restrict__ yval, int64_t* count,
                          const int32_t* __restrict__ colptr, int32_t* xidx, T* xval, LoopState* st,
                          unsigned long long loop) {
    const int64_t ny = count[2];
    const T damping = (T)st->p0;
    const T eps = (T)st->p1;
    T* rank = (T*)st->out;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ny; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = yidx[t];
        const T v = damping * yval[t];
        rank[i] += v;
        if (fabs((double)v) >= (double)eps) {
            const int64_t q = (int64_t)atomicAdd((unsigned long long*)(count + 1), 1ull);
            xidx[q] = i;
            xval[q] = scaled(v, colptr, i);
        }
    }
    if (last_block(&st->ticket) && threadIdx.x == 0) {
        const int64_t kept = *(volatile int64_t*)(count + 1);
        count[0] = kept;
        count[1] = 0;
        const int64_t it = st->iter + 1;
        st->iter = it;
        cudaGraphSetConditional((cudaGraphConditionalHandle)loop, (kept > 0 && it < st->max_iter) ? 1u : 0u);
    }
}

void launch_pr_init(int32_t dtype, int64_t n, double damping, double eps, int32_t max_iter, void* rank,
                    const int32_t* colptr, int32_t* xidx, void* xval, int64_t* count, LoopState* st, int grid,
                    cudaStream_t s) {
    const double c = (1.0 - damping) / (double)n;
    if (dtype == ASV_F64)
        k_pr_init<double><<<grid, 256, 0, s>>>(n, c, damping, eps, max_iter, (double*)rank, colptr, xidx,
                                               (double*)xval, count, st);
    else
        k_pr_init<float><<<grid, 256, 0, s>>>(n, (float)c, damping, eps, max_iter, (float*)rank, colptr, xidx,
                                              (float*)xval, count, st);
}

void launch_pr_step(int32_t dtype, const int32_t* yidx, const void* yval, int64_t* count, const int32_t* colptr,
                    int32_t* xidx, void* xval, LoopState* st, unsigned long long loop, int grid, cudaStream_t s) {
    if (dtype == ASV_F64)
        k_pr_step<double><<<grid, 256, 0, s>>>(yidx, (const double*)yval, count, colptr, xidx, (double*)xval, st,
                                               loop);
    else
        k_pr_step<float><<<grid, 256, 0, s>>>(yidx, (const float*)yval, count, colptr, xidx, (float*)xval, st,
                                              loop);
}

}  // namespace asv
