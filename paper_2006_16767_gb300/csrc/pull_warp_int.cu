// Instantiations of the (sub-)warp row-major kernel for int32 and Boolean.
#include "pull_warp.cuh"

namespace asv {
ASV_INSTANTIATE_PULL_WARP(int32_t)
ASV_INSTANTIATE_PULL_WARP(bool8)

void launch_pull_bool_fused(asv_matrix_s* H, const PullArg& a, bool masked, bool vec, cudaStream_t s) {
    const unsigned lblocks = (unsigned)((H->nseg + 3) / 4);
    const unsigned g = lblocks + (unsigned)((H->m + 128 * kBoolRows - 1) / (128 * kBoolRows));
#define FUSED(MK, V)                                                                                          \
    k_pull_bool_fused<MK, V><<<g, 128, 0, s>>>(H->m, H->nseg, H->nnz, lblocks, H->rowptr, H->seg, H->col, a,  \
                                                H->ws.ywork, H->ws.yflag, H->long_rest, H->long_rest_n)
    if (masked) {
        if (vec) FUSED(true, true);
        else FUSED(true, false);
    } else {
        if (vec) FUSED(false, true);
        else FUSED(false, false);
    }
#undef FUSED
    const unsigned gr = (unsigned)H->num_sms * 4;
#define REST(MK, V)                                                                                            \
    k_pull_long_rest<bool8, MK, V><<<gr, 256, 0, s>>>(H->long_rest, H->long_rest_n, H->nnz, H->col, a, H->ws.ywork, \
                                                      H->ws.yflag)
    if (masked) {
        if (vec) REST(true, true);
        else REST(true, false);
    } else {
        if (vec) REST(false, true);
        else REST(false, false);
    }
#undef REST
}
}  // namespace asv
