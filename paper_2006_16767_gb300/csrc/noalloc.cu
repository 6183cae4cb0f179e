// y = A x for caller-owned CSR arrays without any device allocation.
//
// Some callers cannot call cudaMalloc on their call path: real-time loops in
// which an allocation (or the free that follows it) would synchronise the
// device, runtimes that hand all device memory to their own pool when they
// start, and one-off products on borrowed arrays for which building a
// handle -- which allocates the CSC view and workspaces -- is not an option.
// This entry point serves them with the balanced (merge-path) FP32 SpMV of
// the handle path; its only scratch memory (the tile table and the carries of
// rows that span tiles) lives in a fixed-size array in this file.
#include <mutex>

#include "internal.h"

namespace {

constexpr int64_t kNoAllocMaxTiles = (int64_t)1 << 18;  // m + nnz <= 2^18 * 2048 = 2^29
constexpr size_t kCarryValBytes = 8 * (size_t)kNoAllocMaxTiles;
constexpr size_t kCarryRowBytes = 4 * (size_t)kNoAllocMaxTiles;
constexpr size_t kTileRowBytes = 4 * ((size_t)kNoAllocMaxTiles + 1);
constexpr size_t kScratchBytes = kCarryValBytes + kCarryRowBytes + ((kTileRowBytes + 255) & ~(size_t)255);

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {nullptr};

// Device address of the array on the current device (host code only sees a
// stand-in symbol), looked up once per device and kept for the life of the
// process: a cudaDeviceReset reloads the module and may move the array, so
// this entry point must not be used on a device after it has been reset.
cudaError_t scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = (unsigned char*)p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" asv_status asv_spmv_noalloc_f32(int64_t m, int64_t n, int64_t nnz, const int32_t* d_rowptr,
                                           const int32_t* d_colidx, const float* d_val, const float* d_x,
                                           float* d_y, void* stream) {
    if (m < 0 || n < 0 || nnz < 0) return ASV_ERR_ARG;
    if (m >= INT32_MAX || n >= INT32_MAX || nnz >= INT32_MAX) return ASV_ERR_OVERFLOW;
    if (m == 0) return ASV_OK;
    if (!d_rowptr || !d_y || (nnz > 0 && (!d_colidx || !d_x))) return ASV_ERR_ARG;
    const int64_t D = asv::pull_tile_items(ASV_F32);
    const int64_t ntiles = (m + nnz + D - 1) / D;
    if (ntiles > kNoAllocMaxTiles) return ASV_ERR_CAPACITY;
    unsigned char* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return ASV_ERR_CUDA;
    double* carry_val = (double*)base;
    int32_t* carry_row = (int32_t*)(base + kCarryValBytes);
    int32_t* tile_row = (int32_t*)(base + kCarryValBytes + kCarryRowBytes);
    cudaStream_t s = (cudaStream_t)stream;
    // every tile entry and carry used below is rewritten by this call, so
    // nothing left from an earlier call needs clearing
    asv::launch_partition_raw(d_rowptr, m, nnz, ntiles, tile_row, s);
    // the arrays are not validated; the kernel's bounds checks keep every
    // access inside them even when they are not a valid CSR
    asv::launch_pull_bal_f32_raw(m, n, nnz, d_rowptr, d_colidx, d_val, d_x, d_y, tile_row, carry_row, carry_val, ntiles,
                                 s);
    e = cudaGetLastError();
    return e == cudaSuccess ? ASV_OK : ASV_ERR_CUDA;
}
