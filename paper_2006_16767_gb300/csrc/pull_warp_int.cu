// Instantiations of the (sub-)warp row-major kernel for int32 and Boolean.
#include "pull_warp.cuh"

namespace asv {
ASV_INSTANTIATE_PULL_WARP(int32_t)
ASV_INSTANTIATE_PULL_WARP(bool8)
}  // namespace asv
