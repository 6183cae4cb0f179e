// Definitions shared by the row-major (pull) kernels.
#pragma once
#include <type_traits>

#include "internal.h"
#include "prims.cuh"

namespace asv {

template <class T>
__device__ __forceinline__ T __int_as_float_t(int v) {
    if constexpr (sizeof(T) == 4 && std::is_same<T, float>::value) return __int_as_float(v);
    else return (T)v;
}

struct PullArg {
    const CallDesc* desc;  // read x/y from the call descriptor when non-null
    PullIO io;             // otherwise the pointers given directly
};

__device__ __forceinline__ PullIO resolve(const PullArg& a, void* ywork, bool sparse_out) {
    if (a.desc) {
        PullIO p;
        p.x = a.desc->x_dense;
        p.xbits = a.desc->xbits;
        p.y = sparse_out ? ywork : a.desc->y;
        p.ymask = a.desc->ymask;
        return p;
    }
    return a.io;
}


}  // namespace asv
