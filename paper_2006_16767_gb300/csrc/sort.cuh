// Host launcher of the stable LSD radix sort (8-bit digits) over 32-bit keys.
#pragma once
#include "internal.h"
#include "prims.cuh"

namespace asv {

// Sorts k[0] (and payload v[0] when HAS_V) by the low `key_bits` bits,
// ping-ponging with k[1]/v[1]; returns the index of the buffer that holds the
// result. n may live on the device (n_d). hist needs 256*G+1 ints, blk G+1.
template <class V, bool HAS_V>
int radix_sort(uint32_t* k[2], V* v[2], int64_t n_h, const int64_t* n_d, int key_bits, int32_t* hist,
               int32_t* blk, int G, cudaStream_t s) {
    int cur = 0;
    for (int shift = 0; shift < key_bits; shift += 8) {
        k_radix_hist<256><<<G, 256, 0, s>>>(k[cur], n_h, n_d, shift, hist);
        scan_excl(hist, hist, (int64_t)256 * G, nullptr, blk, G, false, s);
        k_radix_scatter<256, V, HAS_V><<<G, 256, 0, s>>>(k[cur], v[cur], k[cur ^ 1], v[cur ^ 1], n_h, n_d,
                                                         shift, hist);
        cur ^= 1;
    }
    return cur;
}

}  // namespace asv
