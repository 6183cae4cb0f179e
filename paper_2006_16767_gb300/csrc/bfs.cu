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
