// Shared device-side definitions of the adaptive SpMV/SpMSpV library (sm_103a).
#pragma once
#include <type_traits>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/asv.h"

namespace asv {

constexpr int kWarp = 32;

// ---------------------------------------------------------------- value semirings
// bool8 is the storage type of the Boolean (OR, AND) semiring: uint8 0/1, with
// a pattern-only matrix (every stored entry is "1").
typedef uint8_t bool8;

// Neumaier's compensated summation in FP32: the running sum s plus a
// separately accumulated rounding-error term c. The result s + c is within
// about 2u of the exact sum of the addends regardless of their number, which
// keeps FP32 rows with 1e5 entries inside a 2e-6 relative tolerance.
struct KahanF {
    float s, c;
    __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void add(float p) {
        float t = __fadd_rn(s, p);
        float e = (fabsf(s) >= fabsf(p)) ? __fadd_rn(__fsub_rn(s, t), p)
                                          : __fadd_rn(__fsub_rn(p, t), s);
        c = __fadd_rn(c, e);
        s = t;
    }
    __device__ __forceinline__ float value() const { return __fadd_rn(s, c); }
};

// Per-dtype operations. `Acc` accumulates a row in the pull kernels; `Part`
// is the value that crosses lanes/threads; `Atom` is the element type of the
// push-side accumulator array.
template <class T> struct Sr;

template <> struct Sr<float> {
    using Acc = KahanF;
    using Part = float;
    using Atom = double;
    static constexpr bool kPattern = false;
    __device__ __forceinline__ static float mul(float a, float x) { return __fmul_rn(a, x); }
    __device__ __forceinline__ static bool nz(float x) { return x != 0.0f; }
    __device__ __forceinline__ static void acc_zero(Acc& a) { a.zero(); }
    __device__ __forceinline__ static void acc_add(Acc& a, float p) { a.add(p); }
    __device__ __forceinline__ static float acc_val(const Acc& a) { return a.value(); }
    __device__ __forceinline__ static float part_add(float a, float b) { return __fadd_rn(a, b); }
    __device__ __forceinline__ static float acc_part(const Acc& a) { return a.value(); }
    __device__ __forceinline__ static float part_T(float p) { return p; }
    __device__ __forceinline__ static float part_of(float p) { return p; }
    __device__ __forceinline__ static float from_atom(double v) { return __double2float_rn(v); }
    __device__ __forceinline__ static double to_atom(float v) { return (double)v; }
    __device__ __forceinline__ static float one() { return 1.0f; }
};

template <> struct Sr<double> {
    using Acc = double;
    using Part = double;
    using Atom = double;
    static constexpr bool kPattern = false;
    __device__ __forceinline__ static double mul(double a, double x) { return __dmul_rn(a, x); }
    __device__ __forceinline__ static bool nz(double x) { return x != 0.0; }
    __device__ __forceinline__ static void acc_zero(Acc& a) { a = 0.0; }
    __device__ __forceinline__ static void acc_add(Acc& a, double p) { a = __dadd_rn(a, p); }
    __device__ __forceinline__ static double acc_val(const Acc& a) { return a; }
    __device__ __forceinline__ static double part_add(double a, double b) { return __dadd_rn(a, b); }
    __device__ __forceinline__ static double acc_part(const Acc& a) { return a; }
    __device__ __forceinline__ static double part_T(double p) { return p; }
    __device__ __forceinline__ static double part_of(double p) { return p; }
    __device__ __forceinline__ static double from_atom(double v) { return v; }
    __device__ __forceinline__ static double to_atom(double v) { return v; }
    __device__ __forceinline__ static double one() { return 1.0; }
};

// 32-bit two's-complement (+, x): computed in uint32 so wrap-around is defined.
template <> struct Sr<int32_t> {
    using Acc = uint32_t;
    using Part = uint32_t;
    using Atom = uint32_t;
    static constexpr bool kPattern = false;
    __device__ __forceinline__ static uint32_t mul(int32_t a, int32_t x) { return (uint32_t)a * (uint32_t)x; }
    __device__ __forceinline__ static bool nz(int32_t x) { return x != 0; }
    __device__ __forceinline__ static void acc_zero(Acc& a) { a = 0u; }
    __device__ __forceinline__ static void acc_add(Acc& a, uint32_t p) { a += p; }
    __device__ __forceinline__ static int32_t acc_val(const Acc& a) { return (int32_t)a; }
    __device__ __forceinline__ static uint32_t part_add(uint32_t a, uint32_t b) { return a + b; }
    __device__ __forceinline__ static uint32_t acc_part(const Acc& a) { return a; }
    __device__ __forceinline__ static int32_t part_T(uint32_t p) { return (int32_t)p; }
    __device__ __forceinline__ static uint32_t part_of(int32_t v) { return (uint32_t)v; }
    __device__ __forceinline__ static int32_t from_atom(uint32_t v) { return (int32_t)v; }
    __device__ __forceinline__ static uint32_t to_atom(uint32_t v) { return v; }
    __device__ __forceinline__ static int32_t one() { return 1; }
};

// (OR, AND) over a pattern matrix: a_ij = 1 for stored entries, so the product
// is x_j's truth value and the sum is OR.
template <> struct Sr<bool8> {
    using Acc = uint32_t;
    using Part = uint32_t;
    using Atom = uint32_t;
    static constexpr bool kPattern = true;
    __device__ __forceinline__ static uint32_t mul(bool8, bool8 x) { return x != 0; }
    __device__ __forceinline__ static bool nz(bool8 x) { return x != 0; }
    __device__ __forceinline__ static void acc_zero(Acc& a) { a = 0u; }
    __device__ __forceinline__ static void acc_add(Acc& a, uint32_t p) { a |= p; }
    __device__ __forceinline__ static bool8 acc_val(const Acc& a) { return a ? 1 : 0; }
    __device__ __forceinline__ static uint32_t part_add(uint32_t a, uint32_t b) { return a | b; }
    __device__ __forceinline__ static uint32_t acc_part(const Acc& a) { return a; }
    __device__ __forceinline__ static bool8 part_T(uint32_t p) { return p ? 1 : 0; }
    __device__ __forceinline__ static uint32_t part_of(bool8 v) { return v != 0; }
    __device__ __forceinline__ static bool8 from_atom(uint32_t v) { return v ? 1 : 0; }
    __device__ __forceinline__ static uint32_t to_atom(uint32_t v) { return v; }
    __device__ __forceinline__ static bool8 one() { return 1; }
};

// Loads a matrix value; pattern matrices (val == nullptr) read as one.
template <class T>
__device__ __forceinline__ T load_val(const T* val, int64_t k) {
    if (Sr<T>::kPattern || val == nullptr) return Sr<T>::one();
    return __ldg(val + k);
}

// ---------------------------------------------------------------- warp helpers
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

template <class P>
__device__ __forceinline__ P shfl_xor(P v, int mask, int width = 32) {
    return __shfl_xor_sync(0xffffffffu, v, mask, width);
}

template <class P>
__device__ __forceinline__ P shfl_up(P v, int d) {
    return __shfl_up_sync(0xffffffffu, v, d);
}

__device__ __forceinline__ bool test_bit(const uint32_t* bits, int64_t j) {
    return (__ldg(bits + (j >> 5)) >> (j & 31)) & 1u;
}

// The (OR, AND) term of an entry in column c: x_c's truth value. A Boolean x
// is true exactly where its bitmap bit is set, so with the bitmap at hand one
// gather (of a bit: the bitmap is 8x smaller than the byte vector) gives both
// the product and the entry's structural hit, masked or not.
__device__ __forceinline__ uint32_t bool_gather(const bool8* __restrict__ x, const uint32_t* __restrict__ xbits,
                                                int64_t c) {
    return xbits ? (uint32_t)test_bit(xbits, c) : (uint32_t)(__ldg(x + c) != 0);
}

// Sets bit i of a zero-invariant bitmap; the plain read first avoids the
// atomic when the bit is already set (the common case for hub rows).
__device__ __forceinline__ void set_bit_once(uint32_t* bits, int64_t i) {
    uint32_t m = 1u << (i & 31);
    uint32_t* w = bits + (i >> 5);
    if (!(*(volatile uint32_t*)w & m)) atomicOr(w, m);
}

// ---------------------------------------------------------------- per-call descriptor
// Written on the device by the vector-feature pass at the start of every
// selector-driven call, read by every kernel that follows it. Keeping the
// call's pointers and device-side counts here lets one captured CUDA graph
// serve every call on a handle with no host round-trip.
struct CallDesc {
    const void* x_dense;     // dense x the pull kernels read (user's, or the scatter workspace)
    const uint32_t* xbits;   // bitmap of x's structural nonzeros (masked pull)
    const int32_t* xidx;     // x list the push kernels read (user's, or the compaction buffer)
    const void* xval;        // list values, nullptr = ones
    int64_t nnz_x;           // |nz(x)|
    int64_t nnz_s;           // effective nonzeros of A
    void* y;                 // dense output (ASV_OUT_DENSE)
    int32_t* yidx;           // sparse output indices
    void* yval;              // sparse output values
    int64_t* nnz_y;          // sparse output count (device)
    int64_t y_cap;
    const void* user_x_dense;  // the caller's dense x (nullptr when x arrived sparse)
    const int32_t* user_xidx;  // the caller's list (nullptr when x arrived dense)
    const void* user_xval;
    int32_t out_mode;
    int32_t x_sparse;        // 1 when x arrived as a list
    int32_t kid;             // kernel chosen for this call
    int32_t x_ident;         // 1: the list is every column in order (xidx[t] = t), so the
                             // pull kernels read its values in place (x_dense = xval)
    double vfeat[4];         // nnz_x, x_sparsity, nnz_s, m_sparsity
    const uint32_t* ymask;   // output mask: bit i set = row i excluded from y (NULL = none)
    int64_t nhub;            // listed columns longer than kLongSeg (hubs of the thread/warp push)
    int32_t y_ident;         // 1: the list output is every row in order (x reaches every column,
                             // no row is empty, no mask): the pull kernels write its values in
                             // place and the compaction only writes the indices
    int32_t pad;
};

// Predicate of a kernel in one of the selector graph's direct candidate
// chains, which run beside the SWITCH node rather than inside it: such a
// kernel does its work only if the feature pass chose `kid` for the call,
// and otherwise returns at once. kid < 0 (every other launch): always runs.
struct Gate {
    const CallDesc* desc;
    int32_t kid;
    __device__ __forceinline__ bool off() const {
        return kid >= 0 && *(volatile const int32_t*)&desc->kid != kid;
    }
};

// When the two launches of an ordered compaction return at once: a flag set
// (flag != NULL and *flag != 0), or a device count below a bound (count !=
// NULL and *count < below).
struct CompactSkip {
    const int32_t* flag = nullptr;
    const int64_t* count = nullptr;
    int64_t below = 0;
    __device__ __forceinline__ bool on() const { return (flag && *flag) || (count && *count < below); }
};

// Row i is excluded by the output mask.
__device__ __forceinline__ bool row_masked(const uint32_t* __restrict__ ymask, int64_t i) {
    return ymask != nullptr && ((__ldg(ymask + (i >> 5)) >> (i & 31)) & 1u);
}

// Device-resident matrix features (Table 1), written once at handle creation.
struct MatFeat {
    int64_t m, n, nnz, max_row, min_row;
    double avg_row, relative_range, var_nnz_row, gini;
};

// Decision-tree node: feature < 0 marks a leaf whose class is `leaf`.
struct TreeNode {
    int32_t feature;
    int32_t left, right, leaf;
    double thr;
};
constexpr int kMaxTreeNodes = 2048;  // node table of a handle (all formats' trees)
constexpr int kTreeWindow = 1024;    // nodes of one call format staged in shared memory

// Rows longer than kLongRow entries are taken out of the one-row-per-thread
// and sub-warp pull kernels and summed by a warp per segment of at most
// kLongSeg entries (a list built once per matrix): a thread walking a
// power-law hub row of 10^5 entries alone would serialise the whole call.
constexpr int kLongRow = 256;
// Rows of at most kNarrowRow entries let an FP32 push accumulate in FP32:
// kNarrowRow * 2^-24 < 2e-6 (the FP32 tolerance relative to sum |a_ij x_j|).
constexpr int kNarrowRow = 32;
constexpr int kLongSeg = 4096;

// Handle workspaces, passed by value to the kernels that use them.
struct Ws {
    uint32_t* xbits_dense;   // n bits, rewritten by every dense-x feature pass
    uint32_t* xbits_scat;    // n bits, zero-invariant (sparse x -> bitmap)
    void* xdense;            // n values, zero-invariant (sparse x -> dense)
    int32_t* xlist_idx;      // n entries (dense x -> list)
    void* xlist_val;         // n values
    int32_t* xscan;          // n+1 exclusive scan of listed column lengths
    void* acc;               // m 8-byte accumulators, zero-invariant
    uint8_t* yflag;          // m bytes (padded to whole 512-byte groups), zero-invariant: rows in the
                             // structural output set
    void* ywork;             // m values (pull kernels' dense y in sparse-output mode)
    uint32_t* pkeys[2];      // pair buffers for sort / privatised write-back
    void* pvals[2];
    int64_t pair_cap;
    int32_t* hist;           // radix histogram scratch
    int32_t* blk;            // block-count scratch for scans/compaction
    int32_t* status;         // latched device status word
    unsigned long long* counters;  // zero-invariant accumulators of the feature pass
    unsigned int* ticket;    // last-block tickets (zero-invariant)
    // listed columns over kLongSeg entries met by the thread/warp push: list
    // index and a segment cursor per entry, their count; reset to zero by
    // the next call's feature pass
    int2* lcol;
    unsigned int* lcol_n;
    int32_t lcol_cap;
    int32_t* chunk_t0;       // list entry owning the first item of each balanced push chunk
};

__device__ __forceinline__ void latch_status(int32_t* status, int32_t code) {
    if (status) atomicCAS(status, 0, code);
}

}  // namespace asv
